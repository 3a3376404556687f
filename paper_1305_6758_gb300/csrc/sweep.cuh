// Shared-memory checkerboard sweep of many independent simulation paths.
//
// What one path computes (Sec. 2.2 of Rakic et al.): a random initial state,
// then n_therm + n_meas lattice sweeps of Metropolis single spin-flip updates
// of the Heisenberg energy, Eq. (1) plus a Zeeman term -h sum S^z, with unit
// spins of Eq. (2); after every measurement sweep the per-site energy and
// total spin enter FP64 running sums, and the path's outputs are their means
// plus the final state.
//
// GB300 mapping: every path's lattice lives in shared memory for the whole
// run (no HBM traffic per sweep).  A persistent CTA pulls work items from an
// atomic queue; an item is `count` paths of one system, each run by its own
// group of `tp` threads with its own named barrier.  A sweep is two
// half-sweeps: all sites of colour (x+y+z) mod 2 = 0, then all of colour 1.
// Sites of one colour have neighbours only of the other colour, so they
// update independently (this replaces the paper's N randomly chosen sites by
// the checkerboard order; both leave the Boltzmann distribution invariant).
// The colour-1 pass sees final colour-0 neighbours, so the sum over colour-1
// sites of S_i . h_loc,i visits every bond once: the energy comes for free.
//
// Shared-memory layout of one path: [colour][component][half index], the half
// index of site i = x + L(y + Lz) being i >> 1, so a warp's 32 consecutive
// sites of one colour and their +-y, +-z neighbours are 32 consecutive words.
#pragma once
#include <cstdint>

#include "common.cuh"
#include "philox.cuh"

namespace mpk {

// ------------------------------------------------------------ arithmetic --
template <typename Real>
struct Arith;

// FP32 form: 23-bit uniforms (exact in float, open interval), hardware
// approximations for rsqrt, sin/cos and exp.  |S'| = 1 to about 1e-6.
template <>
struct Arith<float> {
  static __device__ __forceinline__ float uni(uint32_t r) {
    return __uint2float_rn((r >> 8) | 1u) * 0x1p-24f;
  }
  // Trial direction uniform on the sphere: cos(theta) = 2u0 - 1, phi = 2 pi u1.
  static __device__ __forceinline__ void trial(uint32_t r0, uint32_t r1, float& x, float& y,
                                               float& z) {
    z = fmaf(2.0f, uni(r0), -1.0f);
    const float q = (1.0f - z) * (1.0f + z);
    const float rad = q * rsqrtf(q);  // q > 0: z never reaches +-1
    float s, c;
    // phi - pi lies in (-pi, pi), where the hardware sin/cos are accurate;
    // cos(phi) = -cos(phi - pi), sin(phi) = -sin(phi - pi).
    __sincosf(6.28318530717958648f * (uni(r1) - 0.5f), &s, &c);
    x = -rad * c;
    y = -rad * s;
  }
  static __device__ __forceinline__ void init_angles(uint32_t r0, uint32_t r1, float& x, float& y,
                                                     float& z) {
    float st, ct, sp, cp;
    sincospif(uni(r0), &st, &ct);
    sincospif(2.0f * uni(r1), &sp, &cp);
    x = st * cp;
    y = st * sp;
    z = ct;
  }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float delta_e(float dx, float dy, float dz, float hx, float hy,
                                                  float hz, float J, float hf) {
    return -J * (dx * hx + dy * hy + dz * hz) - hf * dz;
  }
  static __device__ __forceinline__ bool accept(float dE, float beta, uint32_t r2) {
    return dE <= 0.0f || uni(r2) < __expf(-beta * dE);
  }
  static __device__ __forceinline__ float shfl(float v, int o) {
    return __shfl_xor_sync(0xffffffffu, v, o);
  }
};

// FP64 form: 32-bit uniforms (r + 1/2) 2^-32, IEEE sqrt, library sin/cos/exp,
// and the local-field dot product rounded term by term in the order
// ((dx hx + dy hy) + dz hz) with no fused multiply-add, so that dE matches a
// plain FP64 evaluation bit for bit.
template <>
struct Arith<double> {
  static __device__ __forceinline__ double uni(uint32_t r) {
    return (static_cast<double>(r) + 0.5) * 0x1p-32;
  }
  static __device__ __forceinline__ void trial(uint32_t r0, uint32_t r1, double& x, double& y,
                                               double& z) {
    z = 2.0 * uni(r0) - 1.0;
    const double rad = sqrt(__dmul_rn(1.0 - z, 1.0 + z));
    const double phi = __dmul_rn(2.0 * 3.141592653589793, uni(r1));
    double s, c;
    sincos(phi, &s, &c);
    x = __dmul_rn(rad, c);
    y = __dmul_rn(rad, s);
  }
  static __device__ __forceinline__ void init_angles(uint32_t r0, uint32_t r1, double& x,
                                                     double& y, double& z) {
    const double th = __dmul_rn(3.141592653589793, uni(r0));
    const double ph = __dmul_rn(2.0 * 3.141592653589793, uni(r1));
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    x = __dmul_rn(st, cp);
    y = __dmul_rn(st, sp);
    z = ct;
  }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double delta_e(double dx, double dy, double dz, double hx,
                                                   double hy, double hz, double J, double hf) {
    const double dot = __dadd_rn(__dadd_rn(__dmul_rn(dx, hx), __dmul_rn(dy, hy)), __dmul_rn(dz, hz));
    return __dsub_rn(__dmul_rn(-J, dot), __dmul_rn(hf, dz));
  }
  static __device__ __forceinline__ bool accept(double dE, double beta, uint32_t r2) {
    return dE <= 0.0 || uni(r2) < exp(__dmul_rn(-beta, dE));
  }
  static __device__ __forceinline__ double shfl(double v, int o) {
    return __shfl_xor_sync(0xffffffffu, v, o);
  }
};

// -------------------------------------------------------------- geometry --
// Periodic simple cubic lattice with compile-time L (even).  site() returns
// the site index of half index h in colour c and fills the half indices of
// its neighbours in the other colour, in the fixed order +x, -x, +y, -y, +z, -z.
template <int L>
struct GeomSC {
  static constexpr int N = L * L * L;
  static constexpr int NH = N / 2;
  static constexpr int HL = L / 2;
  static constexpr int HP = L * L / 2;
  static constexpr int NNB = 6;
  __device__ __forceinline__ int count(int) const { return NH; }
  __device__ __forceinline__ int site(int h, int c, int* nb, int& nn) const {
    const int hx = h % HL;
    const int t = h / HL;
    const int y = t % L;
    const int z = t / L;
    const int p = (y + z + c) & 1;
    const int x = 2 * hx + p;
    const int hrow = h - hx;
    nb[0] = hrow + ((x + 1 == L) ? 0 : ((x + 1) >> 1));
    nb[1] = hrow + ((x == 0) ? ((L - 1) >> 1) : ((x - 1) >> 1));
    nb[2] = (y == L - 1) ? h - (L - 1) * HL : h + HL;
    nb[3] = (y == 0) ? h + (L - 1) * HL : h - HL;
    nb[4] = (z == L - 1) ? h - (L - 1) * HP : h + HP;
    nb[5] = (z == 0) ? h + (L - 1) * HP : h - HP;
    nn = 6;
    return 2 * h + p;
  }
};

// Open chain of N spins: colour i mod 2, neighbours i-1 then i+1 where they exist.
struct GeomChain {
  int N;
  static constexpr int NNB = 2;
  __device__ __forceinline__ int count(int c) const { return c == 0 ? (N + 1) >> 1 : N >> 1; }
  __device__ __forceinline__ int site(int h, int c, int* nb, int& nn) const {
    const int i = 2 * h + c;
    nn = 0;
    if (i > 0) nb[nn++] = (i - 1) >> 1;
    if (i < N - 1) nb[nn++] = (i + 1) >> 1;
    return i;
  }
};

// ----------------------------------------------------------- group sync --
// tp threads of one path synchronise on their own named barrier (1 + group),
// or with __syncwarp when the path is one warp.
__device__ __forceinline__ void group_sync(int tp, int bar) {
  if (tp == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(tp) : "memory");
  }
}

// ------------------------------------------------------------- one path --
template <typename Real, class Geom>
__device__ __forceinline__ void run_path(const Geom geo, const DevSystem& sy, int sys_idx,
                                         int64_t path, const SweepParams& P, unsigned char* slice,
                                         int tid, int tp, int bar) {
  using A = Arith<Real>;
  double* acc = reinterpret_cast<double*>(slice + slice_acc_offset());
  double* red = reinterpret_cast<double*>(slice + slice_red_offset());
  Real* sp = reinterpret_cast<Real*>(slice + slice_spin_offset(tp));
  const int NHm = sy.NH;
  const uint32_t c2 = static_cast<uint32_t>(path);
  const uint32_t c3u = kTagUpdate | (static_cast<uint32_t>(sys_idx) << 8);
  const uint32_t c3i = kTagInit | (static_cast<uint32_t>(sys_idx) << 8);
  const Real J = static_cast<Real>(sy.J), hf = static_cast<Real>(sy.h);
  const Real beta = static_cast<Real>(sy.beta);
  const int lane = tid & 31, warp = tid >> 5;

  // Random initial state (Sec. 2.2), or the ordered start of Sec. 5.
  for (int c = 0; c < 2; ++c) {
    Real* own = sp + c * 3 * NHm;
    const int cnt = geo.count(c);
    for (int hh = tid; hh < cnt; hh += tp) {
      int nb[Geom::NNB];
      int nn;
      const int i = geo.site(hh, c, nb, nn);
      const Philox4 r = philox4x32_10(static_cast<uint32_t>(i), 0u, c2, c3i, P.k0, P.k1);
      Real x, y, z;
      if (P.init_mode == MP_INIT_ORDERED) {
        x = Real(0);
        y = Real(0);
        z = Real(1);
      } else if (P.init_mode == MP_INIT_ANGLES) {
        A::init_angles(r.x, r.y, x, y, z);
      } else {
        A::trial(r.x, r.y, x, y, z);
      }
      own[hh] = x;
      own[NHm + hh] = y;
      own[2 * NHm + hh] = z;
    }
  }
  if (tid < kAccDoubles) acc[tid] = 0.0;
  group_sync(tp, bar);

  int accepted = 0;
  const int64_t S = P.n_therm + P.n_meas;
  for (int64_t s = 0; s < S; ++s) {
    const bool meas = s >= P.n_therm;
    Real eb = Real(0), mx = Real(0), my = Real(0), mz = Real(0);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      Real* own = sp + c * 3 * NHm;
      const Real* oth = sp + (1 - c) * 3 * NHm;
      const int cnt = geo.count(c);
      for (int hh = tid; hh < cnt; hh += tp) {
        int nb[Geom::NNB];
        int nn;
        const int i = geo.site(hh, c, nb, nn);
        const Philox4 r =
            philox4x32_10(static_cast<uint32_t>(i), static_cast<uint32_t>(s), c2, c3u, P.k0, P.k1);
        Real tx, ty, tz;
        A::trial(r.x, r.y, tx, ty, tz);
        const Real ax = own[hh], ay = own[NHm + hh], az = own[2 * NHm + hh];
        Real hx = Real(0), hy = Real(0), hz = Real(0);
#pragma unroll
        for (int j = 0; j < Geom::NNB; ++j) {
          if (j < nn) {
            hx = A::add(hx, oth[nb[j]]);
            hy = A::add(hy, oth[NHm + nb[j]]);
            hz = A::add(hz, oth[2 * NHm + nb[j]]);
          }
        }
        const Real dE = A::delta_e(tx - ax, ty - ay, tz - az, hx, hy, hz, J, hf);
        Real nx = ax, ny = ay, nz = az;
        if (A::accept(dE, beta, r.z)) {
          own[hh] = tx;
          own[NHm + hh] = ty;
          own[2 * NHm + hh] = tz;
          nx = tx;
          ny = ty;
          nz = tz;
          ++accepted;
        }
        if (meas) {
          mx += nx;
          my += ny;
          mz += nz;
          if (c == 1) eb += nx * hx + ny * hy + nz * hz;
        }
      }
      if (c == 1 && meas) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          eb += A::shfl(eb, o);
          mx += A::shfl(mx, o);
          my += A::shfl(my, o);
          mz += A::shfl(mz, o);
        }
        if (lane == 0) {
          red[warp * kRedSlots + 0] = static_cast<double>(eb);
          red[warp * kRedSlots + 1] = static_cast<double>(mx);
          red[warp * kRedSlots + 2] = static_cast<double>(my);
          red[warp * kRedSlots + 3] = static_cast<double>(mz);
        }
      }
      group_sync(tp, bar);
    }
    if (meas && tid == 0) {
      double E = 0.0, MX = 0.0, MY = 0.0, MZ = 0.0;
      for (int w = 0; w < (tp >> 5); ++w) {
        E += red[w * kRedSlots + 0];
        MX += red[w * kRedSlots + 1];
        MY += red[w * kRedSlots + 2];
        MZ += red[w * kRedSlots + 3];
      }
      const double invN = 1.0 / static_cast<double>(sy.N);
      const double e = (-sy.J * E - sy.h * MZ) * invN;
      const double ex = MX * invN, ey = MY * invN, ez = MZ * invN;
      const double m2 = ex * ex + ey * ey + ez * ez;
      const double m = sqrt(m2);
      acc[MP_R_E] += e;
      acc[MP_R_E2] += e * e;
      acc[MP_R_M] += m;
      acc[MP_R_M2] += m2;
      acc[MP_R_M4] += m2 * m2;
      acc[MP_R_MX] += ex;
      acc[MP_R_MY] += ey;
      acc[MP_R_MZ] += ez;
      acc[MP_R_MZ2] += ez * ez;
      acc[MP_R_AMZ] += fabs(ez);
      acc[MP_R_EM] += e * m;
      acc[MP_R_EMZ] += e * ez;
      acc[MP_R_MMZ] += m * ez;
      if (s == S - 1) {
        acc[MP_R_FMX] = ex;
        acc[MP_R_FMY] = ey;
        acc[MP_R_FMZ] = ez;
        acc[MP_R_FE] = e;
      }
    }
  }

  // Final state: acceptance count and the worst | |S| - 1 |, reduced over the group.
  double worst = 0.0;
  for (int c = 0; c < 2; ++c) {
    const Real* own = sp + c * 3 * NHm;
    for (int hh = tid; hh < geo.count(c); hh += tp) {
      const double x = own[hh], y = own[NHm + hh], z = own[2 * NHm + hh];
      worst = fmax(worst, fabs(sqrt(x * x + y * y + z * z) - 1.0));
    }
  }
  double nacc = static_cast<double>(accepted);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
    worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  }
  if (lane == 0) {
    red[warp * kRedSlots + 0] = nacc;
    red[warp * kRedSlots + 1] = worst;
  }
  group_sync(tp, bar);
  if (tid == 0) {
    double tot = 0.0, wmax = 0.0;
    for (int w = 0; w < (tp >> 5); ++w) {
      tot += red[w * kRedSlots + 0];
      wmax = fmax(wmax, red[w * kRedSlots + 1]);
    }
    double* rec = P.records + (sy.rec_offset + path) * MP_NREC;
    const double inv = 1.0 / static_cast<double>(P.n_meas);
    for (int k = MP_R_E; k <= MP_R_MMZ; ++k) rec[k] = acc[k] * inv;
    for (int k = MP_R_FMX; k <= MP_R_FE; ++k) rec[k] = acc[k];
    rec[MP_R_ACC] = tot / (static_cast<double>(S) * static_cast<double>(sy.N));
    rec[MP_R_NORM] = wmax;
    rec[MP_R_SPARE] = 0.0;
  }
  if (P.spins != nullptr) {
    double* out = P.spins + P.spin_offset[sys_idx] + path * 3 * static_cast<int64_t>(sy.N);
    for (int c = 0; c < 2; ++c) {
      const Real* own = sp + c * 3 * NHm;
      for (int hh = tid; hh < geo.count(c); hh += tp) {
        int nb[Geom::NNB];
        int nn;
        const int i = geo.site(hh, c, nb, nn);
        out[3 * i + 0] = own[hh];
        out[3 * i + 1] = own[NHm + hh];
        out[3 * i + 2] = own[2 * NHm + hh];
      }
    }
  }
  group_sync(tp, bar);  // the slice is reused by the next item
}

// ------------------------------------------------------- persistent loop --
// The compile-time lattice sizes each precision supports in shared memory.
#define MPK_FOR_EACH_L_FP32(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26)
#define MPK_FOR_EACH_L_FP64(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20)

template <typename Real>
__device__ __forceinline__ void dispatch_path(const DevSystem& sy, int sys_idx, int64_t path,
                                              const SweepParams& P, unsigned char* slice, int tid,
                                              int tp, int bar);

// Largest CTA of each precision: the FP64 form needs more than 64 registers.
template <typename Real>
struct CtaLimit {
  static constexpr int value = sizeof(Real) == 8 ? 512 : kMaxCta;
};

template <typename Real>
__global__ void __launch_bounds__(CtaLimit<Real>::value, 1) sweep_kernel(const SweepParams P) {
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
    if (g < it.count) {
      dispatch_path<Real>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes, tid, sy.tp, 1 + g);
    }
  }
}

}  // namespace mpk
