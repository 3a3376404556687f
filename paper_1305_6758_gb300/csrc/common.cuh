// Shared device-side types of the multipath Metropolis library.
#pragma once
#include <cstdint>

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
  int32_t pad;
  int64_t path_begin;   // path id (random-number counter) of the system's path 0
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
};

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
