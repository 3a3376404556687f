// Shared device-side types of the multipath Metropolis library.
#pragma once
#include <cstdint>

#include <vector_types.h>

#include "mp.h"
#include "philox.cuh"

namespace mpk {

constexpr uint32_t kTagUpdate = 0u;  // counter tag of the sweep updates
constexpr uint32_t kTagInit = 1u;    // counter tag of the initial state
constexpr uint32_t kTagIsing = 4u;   // Ising flip tests: tag 4 + colour
constexpr int32_t kTwoStart = 0x100; // or-ed into SweepParams::init_mode (MP_FLAG_TWO_START)

// Start of one path: with the two-start scheme (Sec. 4) the last floor(P/2)
// paths of a system start from the ordered state.
__host__ __device__ inline int path_init_mode(int32_t mode, int64_t path, int64_t n_paths) {
  return ((mode & kTwoStart) && path >= n_paths - n_paths / 2) ? MP_INIT_ORDERED : (mode & 0xff);
}

constexpr int kAccDoubles = 24;      // FP64 per-path accumulators (>= MP_NREC) in shared memory
constexpr int kRedSlots = 4;         // doubles per warp in the per-sweep reduction
constexpr int kMaxCta = 1024;
// Most paths one CTA can hold: one warp each (groups of more than one warp
// are limited to 15 by the named barriers 1..15).
constexpr int kMaxGroups = kMaxCta / 32;

// One system (lattice, size, temperature, couplings) of a batch, with the
// launch shape the planner chose for it.
struct DevSystem {
  int32_t lattice;      // MP_LATTICE_*
  int32_t L;
  int32_t N;            // sites
  int32_t NH;           // sites of the larger colour (ceil(N/2))
  int32_t tp;           // threads per path (multiple of 32)
  int32_t g;            // paths per CTA
  int32_t slice_bytes;  // shared memory per path
  int32_t ring;         // measurement sweeps per half of the partial-sum ring
  double T, J, h, beta;
  int64_t rec_offset;   // global index of this system's path 0
  int64_t n_paths;
  int32_t mode;         // kModeShared / kModeStreamed / kModePair / kModeGlobal
  int32_t unit_K;       // column segments per column of the unit table (below)
  int64_t path_begin;   // path id (random-number counter) of the system's path 0
  int32_t unit_off;     // first entry of the system's column-walk units in SweepParams::units, or -1
  int32_t unit_U;       // column chunk the unit table was made for
};

constexpr int kModeShared = 0;
constexpr int kModeStreamed = 1;
constexpr int kModePair = 2;  // held in the shared memory of the two CTAs of a cluster
constexpr int kModeGlobal = 3;  // updated in place in HBM (too large for a half-plane ring)
// The sweep-kernel variant of batches whose lattices are all updated in place.
constexpr int kGlobalKernel = -5;
// The lattice size held by two-CTA clusters (FP32 simple cubic L = 32: 393 KB
// of spins), and the shared-memory bytes of one CTA's half with its two halo
// planes per colour: 2 colours x (L/2 + 2) planes x L^2/2 sites x 3 values.
constexpr int kPairL = 32;
__host__ __device__ constexpr int pair_spin_bytes(int L, int real) {
  return 2 * (L / 2 + 2) * (L * L / 2) * 3 * real;
}

// A unit of the persistent work queue: `count` consecutive paths of one
// system, run side by side by one CTA (one thread group per path).
struct WorkItem {
  int32_t sys;
  int32_t count;
  int64_t path0;
};

struct SweepParams {
  const DevSystem* systems;
  const WorkItem* items;
  int* queue;             // work counter, zeroed before each launch
  double* records;        // MP_NREC doubles per path, global path order
  double* spins;          // optional final spins, 3N doubles per path
  const int64_t* spin_offset;  // per-system offset (doubles) into spins
  int32_t n_items;
  int32_t init_mode;
  int64_t n_therm, n_meas;
  PhiloxKeys key;         // round keys of the seed
  void* lattice;          // HBM lattices of streamed paths, one per (CTA, group)
  int64_t lattice_stride; // bytes per lattice buffer
  int32_t lattice_groups; // buffers per CTA
  uint32_t test_stall;    // failure injection: streamed paths skip their first bulk copy
  int* error;             // kErrTimeout / kErrCanceled when a path stopped early
  // Resumable runs: sweeps [s_begin, s_end) of the schedule; per-path state
  // (accumulators, acceptance count, spins) in HBM, loaded and/or saved.
  int64_t s_begin, s_end;
  unsigned char* state;
  const int64_t* state_offset;  // bytes, per system
  const int64_t* state_stride;  // bytes per path, per system
  int32_t resume, save;
  const volatile int* cancel;   // host-mapped cancel flag, or nullptr
  const unsigned long long* ising_thr;  // Ising: 10 acceptance thresholds per system
  // Paths held by the two CTAs of a cluster (kModePair): their work items
  // (one path each) and queue counter.  n_pair_items > 0 requires a launch
  // in clusters of two CTAs.
  const WorkItem* pair_items;
  int32_t n_pair_items;
  int* pair_queue;
  // Column-walk units of the simple cubic lattices in shared memory (see
  // column_unit), made by the host for each system's threads per path; a
  // system without one (unit_off < 0) derives its units on the device.
  const int4* units;
};

// ----------------------------------------------------- column-walk plan --
// The shared-memory walk of a simple cubic lattice takes a colour's sites as
// L^2/2 columns of L planes, each cut into K segments of L/K planes that are
// walked in unrolled chunks of U planes.

// Planes of a column segment interleaved by the compiler (independent Philox
// chains), the chunk U: every segment is a whole number of chunks (the
// segment count K is restricted to divisors of L whose segment length L/K is
// a multiple of U), so no site is left to a serial remainder loop.  FP32
// kernels (512-thread CTAs, up to 128 registers per thread): 8 for L = 8 and
// 16 (a whole column at L = 8), 6 for 12, 18 and 24, 4 for 20, 7 for 14, 3 for
// 6, 2 for 10, 22 and 26, 1 for 2 and 4 (whose columns are too short to split
// into chunks).  The mixed-size kernel holds every size's walk in one register
// allocation and takes 3 for 12 and 18, 2 for 14 and 6 for 24.  FP64 kernels
// (64 registers per thread) take one site at a time.  Measured on the
// benchmark layouts: chunks of 2 lose 6% against 4; 8 gains 1% over 4 at
// L = 16, and 16 (a whole column, spill-free) loses 4% against 8; whole
// chunks of 6 gain 6-8% over a runtime unroll of 4 at L = 12, 18, 24; in the
// batch of uneven sizes, 8 at L = 8 and 6 at L = 24 gain 1.3% together, while
// 6 or 4 at L = 12 lose 0.2-1%.
__host__ __device__ constexpr int column_chunk_fp32(int L, bool mixed) {
  return (L == 16 || L == 8)       ? 8
         : (L % 6 == 0 && L >= 12) ? ((mixed && L < 24) ? 3 : 6)
         : L == 20                 ? 4
         : L == 14                 ? (mixed ? 2 : 7)
         : L == 6                  ? 3
         : L <= 4                  ? 1
                                   : 2;
}
__host__ __device__ constexpr int column_chunk(int real_bytes, int L, bool mixed) {
  return real_bytes == 8 ? 1 : column_chunk_fp32(L, mixed);
}

// Column segments per column: the divisor K of L, with segments of whole
// chunks, that spreads the (L^2/2) K units most evenly over the tp threads
// (the smallest such K, for the longest segments).
__host__ __device__ inline int column_segments(int L, int U, int tp) {
  const int HP = L * L / 2;
  int K = 1;
  double best = -1.0;
  for (int k = 1; k <= L; ++k) {
    if (L % k || (L / k) % U) continue;
    const int units = HP * k;
    const double eff = static_cast<double>(units) / (static_cast<double>((units + tp - 1) / tp) * tp);
    if (eff > best + 1e-9) {
      best = eff;
      K = k;
    }
  }
  return K;
}

// Unit u = g HP + col (column col = x/2 + (L/2) y, segment g of planes
// z0 .. z0 + L/K - 1) as the walk of colour 0 needs it: x = half index of its
// first site | (x parity of that site) << 31; y = half index of that site's
// -z neighbour (bits 0..15) | +-x offset of the sites an even number of
// planes into a chunk (signed, bits 16..23) | the same for the others
// (bits 24..31); z, w = +y and -y offsets.  Colour 1 flips the parity and
// swaps the two x offsets.
__host__ __device__ inline int4 column_unit(int L, int K, int u) {
  const int HL = L / 2, HP = L * L / 2, seg = L / K;
  const int g = u / HP, col = u % HP, z0 = g * seg;
  const int hx = col % HL, y = col / HL;
  const int oyp = (y == L - 1) ? -(L - 1) * HL : HL;
  const int oym = (y == 0) ? (L - 1) * HL : -HL;
  const int oxp1 = (hx == HL - 1) ? -(HL - 1) : 1;  // +x offset when x is odd
  const int oxm0 = (hx == 0) ? (HL - 1) : -1;         // -x offset when x is even
  const int pa = (y + z0) & 1;
  const int oxa = pa ? oxp1 : oxm0, oxb = pa ? oxm0 : oxp1;
  const int hh = col + HP * z0;
  const int mz = z0 == 0 ? hh + (L - 1) * HP : hh - HP;
  int4 d;
  d.x = static_cast<int>(static_cast<unsigned>(hh) | (static_cast<unsigned>(pa) << 31));
  d.y = static_cast<int>(static_cast<unsigned>(mz) | (static_cast<unsigned>(oxa & 0xff) << 16) |
                        (static_cast<unsigned>(oxb & 0xff) << 24));
  d.z = oyp;
  d.w = oym;
  return d;
}

constexpr int kErrTimeout = 1;
constexpr int kErrCanceled = 2;
constexpr int kErrLaunch = 3;  // paths for two-CTA clusters in a launch without clusters
constexpr int kStateHeader = 256;  // bytes before a path's spins in its state: acc[24], accepted
constexpr int kCancelPoll = 16;    // sweeps between polls of the cancel flag

// Byte offsets inside one path's shared-memory slice.
// [acc: FP64 accumulators][ring: 2 x R sweeps x warps x kRedSlots partials][spins]
// (ring elements are sized 8 bytes, enough for either precision and for the
// two doubles per warp of the final reduction)
__host__ __device__ constexpr int slice_acc_offset() { return 0; }
__host__ __device__ constexpr int slice_red_offset() { return kAccDoubles * 8; }
__host__ __device__ inline int slice_spin_offset(int tp, int ring) {
  return kAccDoubles * 8 + (2 * ring * (tp / 32) * kRedSlots * 8 + 127) / 128 * 128;
}

}  // namespace mpk

namespace mpk {
static_assert(kAccDoubles >= MP_NREC, "accumulators must hold a whole record");
static_assert(kAccDoubles <= 32, "accumulators are zeroed by the first warp");
}  // namespace mpk
