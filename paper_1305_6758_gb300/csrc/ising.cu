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
// GB300 mapping: a path's spins are bytes in shared memory,
// [colour][half index], half index i >> 1 = x/2 + (L/2) y.  One Philox call
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

// Flip tests of colour c for this thread's strips.  A strip is the four
// sites of colour c in rows 4j .. 4j+3 at one x/2 = hx (strip index
// hx + (L/2) j, which is also the Philox counter: word y mod 4 serves row y).
// Strips are dealt out round by round, so the lanes of a warp hold
// consecutive hx of the same rows and read consecutive bytes.  Along a strip
// the other colour's spin at the site's own half index is an x neighbour of
// the site in row y and the -y neighbour of the site in row y + 1, and the +y
// neighbour of row y is that x neighbour of row y + 1: from the second row
// on, two of the four neighbours are already in registers.
template <bool kMeas, bool kEnergy>
__device__ __forceinline__ void ising_half_sweep(int L, int c, uint32_t sweep, uint32_t c2,
                                                 uint32_t c3, const PhiloxKeys& key,
                                                 int8_t* __restrict__ own,
                                                 const int8_t* __restrict__ oth,
                                                 const unsigned long long* __restrict__ thr,
                                                 int tid, int tp, int& accepted, int& eb, int& ms) {
  const int HL = L >> 1;
  const int strips = HL * ((L + 3) >> 2);
  const PhiloxPrefix pre = philox_prefix(sweep, c2, c3, key);
  for (int t = tid; t < strips; t += tp) {
    const Philox4 r = philox4x32_10(static_cast<uint32_t>(t), pre, key);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    const int j = t / HL;
    const int hx = t - j * HL;
    const int oxp1 = (hx == HL - 1) ? -(HL - 1) : 1;  // +x offset when x is odd
    const int oxm0 = (hx == 0) ? (HL - 1) : -1;         // -x offset when x is even
    const int y0 = 4 * j;
    int hh = hx + HL * y0;
    int o0 = oth[hh];                                         // the site's own half index
    int dn = oth[y0 == 0 ? hh + (L - 1) * HL : hh - HL];      // -y neighbour
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int y = y0 + k;
      if (y < L) {
        const int p = (y + c) & 1;  // x = 2 hx + p
        const int up = oth[y == L - 1 ? hh - (L - 1) * HL : hh + HL];
        // +x and -x are {o0, xo} in either order (integer sum)
        const int hl = o0 + oth[hh + (p ? oxp1 : oxm0)] + up + dn;
        int s = own[hh];
        const unsigned long long th = thr[(s < 0 ? 5 : 0) + ((hl + 4) >> 1)];
        if (static_cast<unsigned long long>(w[k]) < th) {
          s = -s;
          own[hh] = static_cast<int8_t>(s);
          ++accepted;
        }
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

__device__ void run_path_ising(const DevSystem& sy, int sys_idx, int64_t path,
                               const SweepParams& P, unsigned char* slice, int tid, int tp,
                               int bar) {
  const int L = sy.L, N = sy.N, NH = sy.NH;
  unsigned char* base = slice + slice_spin_offset(tp, sy.ring);
  unsigned long long* thr = reinterpret_cast<unsigned long long*>(base);
  int8_t* sp = reinterpret_cast<int8_t*>(base + kThrBytes);
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
  if (P.resume && st) {
    for (int k = tid; k < N; k += tp) sp[k] = st_spins[k];
    if (tid < kAccDoubles) meter.acc[tid] = reinterpret_cast<const double*>(st)[tid];
  } else {
    // random start: the top bit of word 0 of the site's init counter
    for (int i = tid; i < N; i += tp) {
      const int x = i % L, y = i / L;
      const int c = (x + y) & 1;
      int8_t s = 1;
      if (init != MP_INIT_ORDERED) {
        const Philox4 r = philox4x32_10(static_cast<uint32_t>(i), 0u, c2, kTagInit | sys_hi, P.key);
        s = (r.x >> 31) ? -1 : 1;
      }
      sp[c * NH + (i >> 1)] = s;
    }
    if (tid < kAccDoubles) meter.acc[tid] = 0.0;
  }
  const double accepted_before =
      (P.resume && st) ? reinterpret_cast<const double*>(st)[kAccDoubles] : 0.0;
  if (tid == 0) cancel_flag[gidx] = 0;
  group_sync(tp, bar);

  int accepted = 0;
  bool canceled = false;
  const uint32_t c3a = (kTagIsing + 0u) | sys_hi, c3b = (kTagIsing + 1u) | sys_hi;
  for (int64_t s = P.s_begin; s < P.s_end; ++s) {
    const uint32_t sw = static_cast<uint32_t>(s);
    int eb = 0, ms = 0;
    poll_cancel(P, s, tid, &cancel_flag[gidx]);
    const bool meas = s >= P.n_therm;
    if (meas)
      ising_half_sweep<true, false>(L, 0, sw, c2, c3a, P.key, sp, sp + NH, thr, tid, tp, accepted, eb, ms);
    else
      ising_half_sweep<false, false>(L, 0, sw, c2, c3a, P.key, sp, sp + NH, thr, tid, tp, accepted, eb, ms);
    group_sync(tp, bar);
    if (cancel_flag[gidx]) {
      canceled = true;
      break;
    }
    if (!meas) {
      ising_half_sweep<false, false>(L, 1, sw, c2, c3b, P.key, sp + NH, sp, thr, tid, tp, accepted, eb, ms);
      group_sync(tp, bar);
      continue;
    }
    const int64_t j = s - P.n_therm;
    meter.maybe_flush(j);
    ising_half_sweep<true, true>(L, 1, sw, c2, c3b, P.key, sp + NH, sp, thr, tid, tp, accepted, eb, ms);
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
    for (int k = tid; k < N; k += tp) st_spins[k] = sp[k];
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
      out[3 * i + 2] = static_cast<double>(sp[((x + y) & 1) * NH + (i >> 1)]);
    }
  }
  group_sync(tp, bar);  // the slice is reused by the next item
}

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
      run_path_ising(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes, tid, sy.tp, 1 + g);
  }
}

}  // namespace

cudaError_t ising_prepare(int device, int* max_dynamic, int* max_threads) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, ising_kernel);
  if (e != cudaSuccess) return e;
  *max_dynamic = optin - static_cast<int>(fa.sharedSizeBytes);
  *max_threads = fa.maxThreadsPerBlock;
  return cudaFuncSetAttribute(ising_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, *max_dynamic);
}

cudaError_t ising_occupancy(int cta, int smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, ising_kernel, cta, smem);
}

cudaError_t launch_ising(const SweepParams& p, int grid, int cta, int smem, cudaStream_t st) {
  void* args[] = {const_cast<SweepParams*>(&p)};
  return cudaLaunchKernel(reinterpret_cast<const void*>(ising_kernel), dim3(grid), dim3(cta), args,
                          static_cast<size_t>(smem), st);
}

}  // namespace mpk
