// Multipath Metropolis for the square-lattice Ising model (Appendix A of
// Rakic et al.: the same scheme -- many independent paths from random
// starts, each thermalised and measured -- applied to a model with a discrete
// symmetry, checked against the Onsager-Yang solution).
//
// H = -J sum_bonds s_i s_j - h sum_i s_i, s_i = +-1, on a periodic L x L
// lattice (L even), site i = x + L y, colour (x + y) mod 2.  A sweep tests a
// flip of every colour-0 site, then of every colour-1 site:
// dE = 2 s_i (J sum_nb s_j + h), accepted when dE <= 0, else iff
// u < exp(-beta dE) with u = (r + 1/2) 2^-32 for a Philox word r.
//
// GB300 mapping: a path's spins are bytes in shared memory, one array per
// colour of rows -1 .. L (the rows beyond the lattice are copies of rows L-1
// and 0), byte x/2 of row y for site (x, y).  One Philox call
// serves the four sites of one colour in rows 4j .. 4j+3 at one x/2 = hx:
// row y takes word y mod 4 of Philox(hx + (L/2) j, sweep, path,
// (4 + colour) | sys << 8).
// Every dE > 0 that can occur (5 neighbour sums x 2 spin signs) has its
// acceptance turned, on the host and in FP64, into an integer threshold t
// with u < exp(-beta dE)  <=>  r < t,  so the device test is one integer
// compare and the trajectories equal the FP64 definition exactly.  The
// per-sweep energy (from the colour-1 local fields, every bond once) and
// magnetisation are exact integers; they are reduced with integer shuffles
// and enter the FP64 per-path accumulators of the Heisenberg kernels'
// measurement ring, in the same record layout (m_x = m_y = 0, m_z = m).
#include "kernels.h"
#include "sweep.cuh"

namespace mpk {

namespace {

constexpr int kIsingThreads = 1024;
constexpr int kThrBytes = kIsingThrBytes;  // 10 thresholds (uint64) before the path's spins

// Shared-memory layout of one colour: rows -1 .. L of L/2 bytes (half index
// hx = x/2 within a row), where row -1 is a copy of row L-1 and row L a copy of
// row 0, so the +-y neighbours of every site are one row away with no wrap
// test.  The thread that updates a site of row 0 or row L-1 also writes its
// copy; the copies of colour c are read only as neighbours in the next
// half-sweep, after the barrier that ends this one.
__host__ __device__ constexpr int ising_colour_bytes(int L) { return (L / 2) * (L + 2); }

// Flip tests of colour kC for this thread's strips.  A strip is the four
// sites of colour kC in rows 4j .. 4j+3 at one x/2 = hx (strip index
// hx + (L/2) j, which is also the Philox counter: word y mod 4 serves row y).
// Strips are dealt out round by round, so the lanes of a warp hold
// consecutive hx of the same rows and read consecutive bytes.  Row 4j + k has
// x = 2 hx + ((k + kC) & 1), so which x neighbour sits at the site's own half
// index is known per k at compile time.  Along a strip the other colour's spin
// at the site's own half index is an x neighbour of the site in row y and the
// -y neighbour of the site in row y + 1, and the +y neighbour of row y is that
// x neighbour of row y + 1: from the second row on, two of the four
// neighbours are already in registers.  kL > 0: the lattice size is a
// compile-time constant (divisions and offsets become immediates); kL = 0:
// any even L.
template <int kL, int kC, bool kMeas, bool kEnergy>
__device__ __forceinline__ void ising_half_sweep(int Lrt, uint32_t sweep, uint32_t c2, uint32_t c3,
                                                 const PhiloxKeys& key, int8_t* __restrict__ own,
                                                 const int8_t* __restrict__ oth,
                                                 const unsigned long long* __restrict__ thr, int tid,
                                                 int tp, int& accepted, int& eb, int& ms) {
  const int L = kL > 0 ? kL : Lrt;
  const int HL = L >> 1;
  const int strips = HL * ((L + 3) >> 2);
  const PhiloxPrefix pre = philox_prefix(sweep, c2, c3, key);
  for (int t = tid; t < strips; t += tp) {
    const Philox4 r = philox4x32_10(static_cast<uint32_t>(t), pre, key);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    // t >= 0: unsigned division by HL (a compile-time constant for kL > 0)
    const int j = static_cast<int>(static_cast<unsigned>(t) / static_cast<unsigned>(HL));
    const int hx = t - j * HL;
    const int oxp1 = (hx == HL - 1) ? -(HL - 1) : 1;  // +x offset when x is odd
    const int oxm0 = (hx == 0) ? (HL - 1) : -1;         // -x offset when x is even
    int hh = HL * (4 * j + 1) + hx;  // row 4j (row -1 comes first)
    int o0 = oth[hh];                // the site's own half index
    int dn = oth[hh - HL];           // -y neighbour
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int y = 4 * j + k;
      if ((kL > 0 && kL % 4 == 0) || y < L) {
        const int up = oth[hh + HL];
        // +x and -x are {o0, xo} in either order (integer sum)
        const int hl = o0 + oth[hh + (((k + kC) & 1) ? oxp1 : oxm0)] + up + dn;
        int s = own[hh];
        // threshold (s < 0 ? 5 : 0) + (hl + 4) / 2 for s = +-1, hl = -4 .. 4 even
        const unsigned long long th = thr[(hl + 9 - 5 * s) >> 1];
        if (static_cast<unsigned long long>(w[k]) < th) {
          s = -s;
          own[hh] = static_cast<int8_t>(s);
          ++accepted;
        }
        if (k == 0 && j == 0) own[hh + L * HL] = static_cast<int8_t>(s);  // row 0 -> row L
        if (y == L - 1) own[hh - L * HL] = static_cast<int8_t>(s);         // row L-1 -> row -1
        if (kMeas) {
          ms += s;
          if (kEnergy) eb += s * hl;
        }
        dn = o0;
        o0 = up;
        hh += HL;
      }
    }
  }
}

template <int kL>
__device__ void run_path_ising(const DevSystem& sy, int sys_idx, int64_t path,
                               const SweepParams& P, unsigned char* slice, int tid, int tp,
                               int bar) {
  const int L = kL > 0 ? kL : sy.L, N = sy.N, NH = sy.NH, HL = L / 2;
  const int CB = ising_colour_bytes(L);
  unsigned char* base = slice + slice_spin_offset(tp, sy.ring);
  unsigned long long* thr = reinterpret_cast<unsigned long long*>(base);
  int8_t* sp = reinterpret_cast<int8_t*>(base + kThrBytes);
  // byte of site (x, y) in its colour's array, and where its row copy goes
  auto at = [&](int x, int y) { return ((x + y) & 1) * CB + HL * (y + 1) + (x >> 1); };
  const uint32_t c2 = static_cast<uint32_t>(sy.path_begin + path);  // path id
  const uint32_t sys_hi = static_cast<uint32_t>(sys_idx) << 8;
  const int init = path_init_mode(P.init_mode, path, sy.n_paths);
  const int64_t j_first = P.s_begin > P.n_therm ? P.s_begin - P.n_therm : 0;
  Meter<double> meter{reinterpret_cast<double*>(slice + slice_acc_offset()),
                      reinterpret_cast<double*>(slice + slice_red_offset()),
                      sy.ring, tp >> 5, tid & 31, tid >> 5, tid,
                      1.0 / static_cast<double>(N), sy.J, sy.h, j_first};
  meter.start();
  unsigned char* st = path_state(P, sys_idx, path);
  int8_t* st_spins = st ? reinterpret_cast<int8_t*>(st + kStateHeader) : nullptr;
  __shared__ int cancel_flag[kMaxGroups];
  const int gidx = bar - 1;

  if (tid < 10) thr[tid] = P.ising_thr[sys_idx * 10 + tid];
  // initial or saved spins (saved as [colour][half index x/2 + (L/2) y]),
  // with rows 0 and L-1 also written to their copies
  const bool resume = P.resume && st;
  for (int i = tid; i < N; i += tp) {
    const int x = i % L, y = i / L;
    const int c = (x + y) & 1;
    int8_t s = 1;
    if (resume) {
      s = st_spins[c * NH + (i >> 1)];
    } else if (init != MP_INIT_ORDERED) {
      // random start: the top bit of word 0 of the site's init counter
      const Philox4 r = philox4x32_10(static_cast<uint32_t>(i), 0u, c2, kTagInit | sys_hi, P.key);
      s = (r.x >> 31) ? -1 : 1;
    }
    const int b = at(x, y);
    sp[b] = s;
    if (y == 0) sp[b + L * HL] = s;
    if (y == L - 1) sp[b - L * HL] = s;
  }
  if (tid < kAccDoubles) meter.acc[tid] = resume ? reinterpret_cast<const double*>(st)[tid] : 0.0;
  const double accepted_before = resume ? reinterpret_cast<const double*>(st)[kAccDoubles] : 0.0;
  if (tid == 0) cancel_flag[gidx] = 0;
  group_sync(tp, bar);

  int accepted = 0;
  bool canceled = false;
  const uint32_t c3a = (kTagIsing + 0u) | sys_hi, c3b = (kTagIsing + 1u) | sys_hi;
  int8_t* sp0 = sp;
  int8_t* sp1 = sp + CB;
  for (int64_t s = P.s_begin; s < P.s_end; ++s) {
    const uint32_t sw = static_cast<uint32_t>(s);
    int eb = 0, ms = 0;
    poll_cancel(P, s, tid, &cancel_flag[gidx]);
    const bool meas = s >= P.n_therm;
    if (meas)
      ising_half_sweep<kL, 0, true, false>(L, sw, c2, c3a, P.key, sp0, sp1, thr, tid, tp, accepted, eb, ms);
    else
      ising_half_sweep<kL, 0, false, false>(L, sw, c2, c3a, P.key, sp0, sp1, thr, tid, tp, accepted, eb, ms);
    group_sync(tp, bar);
    if (cancel_flag[gidx]) {
      canceled = true;
      break;
    }
    if (!meas) {
      ising_half_sweep<kL, 1, false, false>(L, sw, c2, c3b, P.key, sp1, sp0, thr, tid, tp, accepted, eb, ms);
      group_sync(tp, bar);
      continue;
    }
    const int64_t j = s - P.n_therm;
    meter.maybe_flush(j);
    ising_half_sweep<kL, 1, true, true>(L, sw, c2, c3b, P.key, sp1, sp0, thr, tid, tp, accepted, eb, ms);
    // exact integer partials of this warp, then one slot of the ring
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      eb += __shfl_xor_sync(0xffffffffu, eb, o);
      ms += __shfl_xor_sync(0xffffffffu, ms, o);
    }
    if ((tid & 31) == 0) {
      double* r = meter.cur_slot() + (tid >> 5) * kRedSlots;
      r[0] = static_cast<double>(eb);
      r[1] = 0.0;
      r[2] = 0.0;
      r[3] = static_cast<double>(ms);
    }
    meter.advance();
    group_sync(tp, bar);
  }
  if (canceled) {
    group_sync(tp, bar);
    return;
  }
  const int64_t n_meas_done = P.s_end > P.n_therm ? P.s_end - P.n_therm : 0;
  meter.finish(n_meas_done);
  group_sync(tp, bar);
  if (P.save && st) {
    for (int i = tid; i < N; i += tp) {
      const int x = i % L, y = i / L;
      st_spins[((x + y) & 1) * NH + (i >> 1)] = sp[at(x, y)];
    }
    if (tid < kAccDoubles) reinterpret_cast<double*>(st)[tid] = meter.acc[tid];
  }
  meter.write_record(P.records + (sy.rec_offset + path) * MP_NREC, accepted, 0.0, P.s_end,
                     n_meas_done, N, tp, bar, accepted_before,
                     (P.save && st) ? reinterpret_cast<double*>(st) + kAccDoubles : nullptr);
  if (P.spins != nullptr) {
    double* out = P.spins + P.spin_offset[sys_idx] + path * 3 * static_cast<int64_t>(N);
    for (int i = tid; i < N; i += tp) {
      const int x = i % L, y = i / L;
      out[3 * i + 0] = 0.0;
      out[3 * i + 1] = 0.0;
      out[3 * i + 2] = static_cast<double>(sp[at(x, y)]);
    }
  }
  group_sync(tp, bar);  // the slice is reused by the next item
}

// One kernel per lattice size of the appendix (20, 40, 50, 60: a batch whose
// systems all have that size) and one for any even L.  Separate kernels keep
// each size's register allocation to itself.
template <int kL>
__global__ void __launch_bounds__(kIsingThreads, 1) ising_kernel(const SweepParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(P.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= P.n_items) return;
    const WorkItem it = P.items[item];
    const DevSystem sy = P.systems[it.sys];
    const int g = static_cast<int>(threadIdx.x) / sy.tp;
    const int tid = static_cast<int>(threadIdx.x) - g * sy.tp;
    if (g < it.count)
      run_path_ising<kL>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes, tid, sy.tp, 1 + g);
  }
}

const void* ising_kernel_of(int variant) {
  switch (ising_variant_L(variant)) {
    case 20: return reinterpret_cast<const void*>(ising_kernel<20>);
    case 40: return reinterpret_cast<const void*>(ising_kernel<40>);
    case 50: return reinterpret_cast<const void*>(ising_kernel<50>);
    case 60: return reinterpret_cast<const void*>(ising_kernel<60>);
    default: return reinterpret_cast<const void*>(ising_kernel<0>);
  }
}

}  // namespace

bool ising_compiled_L(int L) { return L == 20 || L == 40 || L == 50 || L == 60; }

cudaError_t ising_prepare(int variant, int device, int* max_dynamic, int* max_threads) {
  const void* k = ising_kernel_of(variant);
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  *max_dynamic = optin - static_cast<int>(fa.sharedSizeBytes);
  *max_threads = fa.maxThreadsPerBlock;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, *max_dynamic);
}

cudaError_t ising_occupancy(int variant, int cta, int smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, ising_kernel_of(variant), cta, smem);
}

cudaError_t launch_ising(int variant, const SweepParams& p, int grid, int cta, int smem, cudaStream_t st) {
  void* args[] = {const_cast<SweepParams*>(&p)};
  return cudaLaunchKernel(ising_kernel_of(variant), dim3(grid), dim3(cta), args, static_cast<size_t>(smem), st);
}

}  // namespace mpk
