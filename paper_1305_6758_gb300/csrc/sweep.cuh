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
// Shared-memory layout of one path: [colour][(x, y) pairs | z][half index],
// the half index of site i = x + L(y + Lz) being i >> 1, so a spin is one
// 8-byte and one 4-byte load (16 + 8 in FP64) and a warp's 32 consecutive
// sites of one colour and their +-y, +-z neighbours are consecutive elements.
#pragma once
#include <cstdint>

#include "common.cuh"
#include "philox.cuh"

namespace mpk {

// ------------------------------------------------------------ arithmetic --
template <typename Real>
struct Arith;

// FP32 form: 23-bit uniforms (exact in float, open interval), hardware
// approximations for rsqrt, sin/cos and 2^x.  |S'| = 1 to about 1e-6.
template <>
struct Arith<float> {
  // 1 + m 2^-23 with m the top 23 bits of r, built from the bits (no int->float
  // conversion); the uniform is that minus (1 - 2^-24) = (2m + 1) 2^-24, exactly.
  static __device__ __forceinline__ float one_plus(uint32_t r) {
    return __uint_as_float(0x3f800000u | (r >> 9));
  }
  static __device__ __forceinline__ float uni(uint32_t r) { return one_plus(r) - 0.99999994f; }
  // Trial direction uniform on the sphere: cos(theta) = 2u0 - 1, phi = 2 pi u1.
  static __device__ __forceinline__ void trial(uint32_t r0, uint32_t r1, float& x, float& y,
                                               float& z) {
    z = fmaf(2.0f, uni(r0), -1.0f);  // 2 u0 - 1, exact, never +-1
    const float q = fmaf(-z, z, 1.0f);  // 1 - z^2 > 0
    const float rad = q * rsqrtf(q);
    float s, c;
    // phi - pi = 2 pi (u1 - 1/2) lies in (-pi, pi), where the hardware sin/cos
    // are accurate; cos(phi) = -cos(phi - pi), sin(phi) = -sin(phi - pi).
    __sincosf(fmaf(6.28318531f, one_plus(r1), -9.42477763f), &s, &c);
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
  // Metropolis test of the move S -> S + d in the local field (hx, hy, hz):
  // accept when dE <= 0, else iff u < exp(-beta dE) = 2^(-x), with
  // x = beta log2(e) dE = (-b J) d.h_loc + (-b h) d_z and b = beta log2(e)
  // precomputed per path (the two products are loop invariants).
  static __device__ __forceinline__ bool accept_move(float dx, float dy, float dz, float hx,
                                                     float hy, float hz, float J, float hf,
                                                     float blog2e, uint32_t r2) {
    const float x = fmaf(-blog2e * J, dx * hx + dy * hy + dz * hz, (-blog2e * hf) * dz);
    float p;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p) : "f"(-x));
    return x <= 0.0f || uni(r2) < p;
  }
  static __device__ __forceinline__ float beta_param(double beta) {
    return static_cast<float>(beta * 1.4426950408889634);
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
  static __device__ __forceinline__ bool accept_move(double dx, double dy, double dz, double hx,
                                                     double hy, double hz, double J, double hf,
                                                     double beta, uint32_t r2) {
    const double dE = delta_e(dx, dy, dz, hx, hy, hz, J, hf);
    return dE <= 0.0 || uni(r2) < exp(__dmul_rn(-beta, dE));
  }
  static __device__ __forceinline__ double beta_param(double beta) { return beta; }
  static __device__ __forceinline__ double shfl(double v, int o) {
    return __shfl_xor_sync(0xffffffffu, v, o);
  }
};

// -------------------------------------------------------------- geometry --
// Periodic simple cubic lattice with compile-time L (even).  site() returns
// the site index of half index h in colour c and fills the half indices of
// its neighbours in the other colour, in the fixed order +x, -x, +y, -y, +z, -z.
// Half index h = hx + HL*y + HP*z with hx = x / 2.  kMixed: the geometry as
// run by the mixed-size kernel (which takes the column-walk chunks of
// column_chunk_fp32(L, true)).
template <int L, bool kMixed = false>
struct GeomSC {
  static constexpr bool kInMixed = kMixed;
  static constexpr int N = L * L * L;
  static constexpr int NH = N / 2;
  static constexpr int HL = L / 2;
  static constexpr int HP = L * L / 2;
  static constexpr int NNB = 6;
  static constexpr bool kColumns = true;
  __device__ __forceinline__ int count(int) const { return NH; }
  static __device__ __forceinline__ constexpr int stride() { return NH; }
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

// Periodic simple cubic lattice of run-time L (even), every site decoded from
// its half index (neighbours in the same fixed order as GeomSC): the geometry
// of lattices updated in place in HBM, which are too large for a ring of
// half-planes in shared memory.
struct GeomSCDyn {
  int L;
  static constexpr int NNB = 6;
  static constexpr bool kColumns = false;
  __device__ __forceinline__ int count(int) const { return L * L * L / 2; }
  __device__ __forceinline__ int stride() const { return L * L * L / 2; }
  __device__ __forceinline__ int site(int h, int c, int* nb, int& nn) const {
    const int HL = L / 2, HP = L * L / 2;
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
  static constexpr bool kColumns = false;
  static constexpr int HP = 1;
  __device__ __forceinline__ int count(int c) const { return c == 0 ? (N + 1) >> 1 : N >> 1; }
  // even, so that every (x, y) pair array starts on a pair boundary
  __device__ __forceinline__ int stride() const { return (((N + 1) >> 1) + 1) & ~1; }
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

// ------------------------------------------------------- one attempt -----
// Per-thread partial sums of the measurement of one sweep.
template <typename Real>
struct Partials {
  Real eb, mx, my, mz;
};

// ------------------------------------------------------------ spin views --
template <typename Real>
struct V3 {
  Real x, y, z;
};
template <typename Real>
__device__ __forceinline__ V3<Real> add3(V3<Real> a, V3<Real> b) {
  using A = Arith<Real>;
  return V3<Real>{A::add(a.x, b.x), A::add(a.y, b.y), A::add(a.z, b.z)};
}
template <typename Real>
struct PairOf;
template <>
struct PairOf<float> {
  using T = float2;
};
template <>
struct PairOf<double> {
  using T = double2;
};

// S spins of one colour (or one half-plane): their (x, y) pairs, then their z
// components.  base must be aligned to a pair and S even.
template <typename Real>
struct SpinView {
  using P2 = typename PairOf<Real>::T;
  P2* xy;
  Real* z;
  __device__ __forceinline__ SpinView(Real* base, int S)
      : xy(reinterpret_cast<P2*>(base)), z(base + 2 * S) {}
  __device__ __forceinline__ V3<Real> ld(int h) const {
    const P2 v = xy[h];
    return V3<Real>{v.x, v.y, z[h]};
  }
  __device__ __forceinline__ void st(int h, Real a, Real b, Real c) const {
    P2 v;
    v.x = a;
    v.y = b;
    xy[h] = v;
    z[h] = c;
  }
};

// The Metropolis step at site i (half index hh of the colour view `own`)
// given its local field (hx, hy, hz), Sec. 2.2: trial spin, energy change
// from the local field, acceptance test.
template <typename Real, bool kMeas, bool kEnergy>
__device__ __forceinline__ void update(uint32_t i, const PhiloxPrefix& pre, const PhiloxKeys& key, const SpinView<Real>& own, int hh,
                                       Real hx, Real hy, Real hz, Real J, Real hf, Real bp,
                                       int& accepted, Partials<Real>& part) {
  using A = Arith<Real>;
  const Philox4 r = philox4x32_10(i, pre, key);
  Real tx, ty, tz;
  A::trial(r.x, r.y, tx, ty, tz);
  const V3<Real> a = own.ld(hh);
  const Real ax = a.x, ay = a.y, az = a.z;
  Real nx = ax, ny = ay, nz = az;
  if (A::accept_move(tx - ax, ty - ay, tz - az, hx, hy, hz, J, hf, bp, r.z)) {
    own.st(hh, tx, ty, tz);
    nx = tx;
    ny = ty;
    nz = tz;
    ++accepted;
  }
  if (kMeas) {
    part.mx += nx;
    part.my += ny;
    part.mz += nz;
    if (kEnergy) part.eb += nx * hx + ny * hy + nz * hz;
  }
}

// One Metropolis attempt with the neighbours' half indices nb[0..nn) in `oth`,
// summed in the fixed order nb[0], nb[1], ...
template <typename Real, int NNB, bool kMeas, bool kEnergy>
__device__ __forceinline__ void attempt(uint32_t i, const PhiloxPrefix& pre, const PhiloxKeys& key, const SpinView<Real>& own,
                                        const SpinView<Real>& oth, int hh, const int* nb, int nn,
                                        Real J, Real hf, Real bp, int& accepted,
                                        Partials<Real>& part) {
  V3<Real> f{Real(0), Real(0), Real(0)};
#pragma unroll
  for (int j = 0; j < NNB; ++j) {
    if (j < nn) f = add3(f, oth.ld(nb[j]));
  }
  update<Real, kMeas, kEnergy>(i, pre, key, own, hh, f.x, f.y, f.z, J, hf, bp, accepted,
                               part);
}

// The column chunk U of a geometry (column_chunk in common.cuh).
template <typename Real, class Geom>
constexpr int kColumnChunk = column_chunk(static_cast<int>(sizeof(Real)), 2 * Geom::HL, Geom::kInMixed);

// One half-sweep of one thread: every site of colour c it owns.
//
// Column-segment walk (simple cubic, K > 0): a colour's sites form L^2/2
// columns col = x/2 + (L/2) y of L planes each (half index col + (L^2/2) z);
// each column is cut into K segments of L/K planes, and the HP * K units
// (column col, segment g), numbered u = g * HP + col, are dealt out to the
// threads round by round (thread tid takes u = tid, tid + tp, ...), so the
// lanes of a warp work on consecutive columns of the same planes and their
// shared-memory accesses are consecutive elements.  A segment is walked in
// chunks of kColumnChunk planes whose sites the compiler interleaves.  Within a segment the +-x
// and +-y neighbour offsets are fixed, and since the x parity flips from
// plane to plane, the other colour's spin at the site's own half index is
// both an x neighbour of the site in plane z and the -z neighbour of the site
// in plane z + 1, while the +z neighbour of one site is an x neighbour of the
// next: after the first site of a segment two of the six neighbours are
// already in registers.  The two x neighbours are added first, in either
// order (a + b = b + a exactly), so the sum keeps the fixed order +x, -x, +y,
// -y, +z, -z.  K = 0: every site decoded from its half index (open chains).
template <typename Real, class Geom, bool kMeas, bool kEnergy>
__device__ __forceinline__ void half_sweep(const Geom& geo, int c, const PhiloxPrefix& pre,
                                           const PhiloxKeys& key, Real* sp, int tid,
                                           int tp, int K, const int4* units, Real J, Real hf, Real bp,
                                           int& accepted, Partials<Real>& part) {
  const int S = geo.stride();
  const SpinView<Real> own(sp + c * 3 * S, S);
  const SpinView<Real> oth(sp + (1 - c) * 3 * S, S);
  if constexpr (Geom::kColumns) {
    if (K > 0) {
      constexpr int HL = Geom::HL, HP = Geom::HP, LL = 2 * Geom::HL;
      const int seg = LL / K;  // planes per segment
      constexpr int U = kColumnChunk<Real, Geom>;
      constexpr int NH = HP * LL;
      for (int u = tid; u < HP * K; u += tp) {
        // the unit: half index hh of its first site and of that site's -z
        // neighbour, +-y offsets, and the x parity p of the site: it flips
        // from plane to plane, so sites an even number of planes after the
        // chunk's first take (pa, oxa), the others (pb, oxb), and within a
        // chunk the choice is made at compile time
        int hh, mzi, oyp, oym, pa, oxa, oxb;
        if (units != nullptr) {  // from the host's table (column_unit)
          const int4 d = __ldg(units + u);
          hh = d.x & 0x7fffffff;
          pa = static_cast<int>(static_cast<unsigned>(d.x) >> 31) ^ c;
          mzi = d.y & 0xffff;
          const int xa = (d.y << 8) >> 24, xb = d.y >> 24;  // signed bytes 2 and 3
          oxa = c ? xb : xa;
          oxb = c ? xa : xb;
          oyp = d.z;
          oym = d.w;
        } else {
          // u >= 0: unsigned division by the compile-time HP and HL needs no
          // sign fix-up
          const unsigned uu = static_cast<unsigned>(u);
          const int g = static_cast<int>(uu / HP);
          const int col = static_cast<int>(uu % HP);
          const int z0 = g * seg;
          const int hx = static_cast<int>(static_cast<unsigned>(col) % HL);
          const int y = static_cast<int>(static_cast<unsigned>(col) / HL);
          oyp = (y == LL - 1) ? -(LL - 1) * HL : HL;
          oym = (y == 0) ? (LL - 1) * HL : -HL;
          const int oxp1 = (hx == HL - 1) ? -(HL - 1) : 1;  // +x offset when x is odd
          const int oxm0 = (hx == 0) ? (HL - 1) : -1;         // -x offset when x is even
          pa = (y + z0 + c) & 1;
          oxa = pa ? oxp1 : oxm0;
          oxb = pa ? oxm0 : oxp1;
          hh = col + HP * z0;
          mzi = z0 == 0 ? hh + (LL - 1) * HP : hh - HP;
        }
        int pb = pa ^ 1;
        const int oxx = oxa ^ oxb;
        V3<Real> o0 = oth.ld(hh);   // the other colour at the site's half index
        V3<Real> mz = oth.ld(mzi);  // -z neighbour
        for (int zc = 0; zc < seg; zc += U) {
#pragma unroll
          for (int k = 0; k < U; ++k, hh += HP) {
            const int p = (k & 1) ? pb : pa;
            const int nxo = hh + ((k & 1) ? oxb : oxa);
            // chunks start at multiples of U, which divides L: only a chunk's
            // last plane can be plane L - 1, whose +z neighbour wraps
            const int zn = (k == U - 1 && hh + HP >= NH) ? hh + HP - NH : hh + HP;
            const V3<Real> cz = oth.ld(zn);
            const V3<Real> f =
                add3(add3(add3(add3(add3(o0, oth.ld(nxo)), oth.ld(hh + oyp)), oth.ld(hh + oym)), cz), mz);
            update<Real, kMeas, kEnergy>(static_cast<uint32_t>(2 * hh + p), pre, key, own, hh,
                                         f.x, f.y, f.z, J, hf, bp, accepted, part);
            mz = o0;
            o0 = cz;
          }
          if constexpr (U & 1) {  // an odd chunk: the next one starts on the other parity
            pa ^= 1;
            pb ^= 1;
            oxa ^= oxx;
            oxb ^= oxx;
          }
        }
      }
      return;
    }
  }
  const int cnt = geo.count(c);
  for (int hh = tid; hh < cnt; hh += tp) {
    int nb[Geom::NNB];
    int nn;
    const int i = geo.site(hh, c, nb, nn);
    attempt<Real, Geom::NNB, kMeas, kEnergy>(static_cast<uint32_t>(i), pre, key, own, oth,
                                             hh, nb, nn, J, hf, bp, accepted, part);
  }
}

// ----------------------------------------------------------- measurement --
// Per-path measurement state in the path's shared-memory slice: the FP64
// accumulators and the partial-sum ring.  ring[half][slot][warp][4] holds each
// warp's partial sums (E_bond, Mx, My, Mz) of one measurement sweep; a half of
// R sweeps is flushed into the FP64 accumulators by all warps together after
// the next barrier while the other half fills, so no warp carries the
// bookkeeping alone and no FP64 operation runs per sweep.
template <typename Real>
struct Meter {
  double* acc;
  Real* red;
  int R, nwarps, lane, warp, tid;
  double invN;
  Real J, hf;
  int64_t j_first;  // first measurement sweep of this call (earlier ones are already flushed)
  // ring slot of the next measurement sweep j to record, ((j / R) & 1) * R +
  // j % R, kept in a 32-bit counter that advances one sweep at a time (no
  // 64-bit division per sweep); start() sets it for j_first
  int cur = 0;
  // partial sums per sweep (one per warp of the path: nwarps, or twice that
  // when two CTAs of a cluster hold the lattice), and the first of them this
  // CTA's warps write (the partner CTA writes into the owner's ring)
  int nslot = 0, slot_off = 0;

  __device__ void start() {
    if (nslot == 0) nslot = nwarps;
    cur = static_cast<int>(((j_first / R) & 1) * R + j_first % R);
  }
  __device__ Real* slot(int64_t j) const {
    return red + ((((j / R) & 1) * R + (j % R)) * nslot) * kRedSlots;
  }
  __device__ Real* cur_slot() const { return red + (cur * nslot) * kRedSlots; }
  __device__ void advance() {
    if (++cur == 2 * R) cur = 0;
  }
  // Per-site observables (Sec. 2.2) of one measurement sweep from its slot.
  __device__ void observe(const Real* sl, Real& e, Real& ex, Real& ey, Real& ez) const {
    Real E = Real(0), MX = Real(0), MY = Real(0), MZ = Real(0);
    for (int w = 0; w < nslot; ++w) {
      E += sl[w * kRedSlots + 0];
      MX += sl[w * kRedSlots + 1];
      MY += sl[w * kRedSlots + 2];
      MZ += sl[w * kRedSlots + 3];
    }
    const Real rN = static_cast<Real>(invN);
    e = (-J * E - hf * MZ) * rN;
    ex = MX * rN;
    ey = MY * rN;
    ez = MZ * rN;
  }
  // Store this warp's partials of the current measurement sweep and move to
  // the next (every lane calls, once per measurement sweep, in order).
  __device__ void record(Partials<Real> part) {
    using A = Arith<Real>;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      part.eb += A::shfl(part.eb, o);
      part.mx += A::shfl(part.mx, o);
      part.my += A::shfl(part.my, o);
      part.mz += A::shfl(part.mz, o);
    }
    if (lane == 0) {
      Real* r = cur_slot() + (slot_off + warp) * kRedSlots;
      r[0] = part.eb;
      r[1] = part.mx;
      r[2] = part.my;
      r[3] = part.mz;
    }
    advance();
  }
  // Flush sweeps j0 .. j0+n-1 (one ring half): lane l takes sweep j0+l; warp
  // w owns observables w, w + warps, ...; each owned observable is summed
  // over the lanes and added to its FP64 accumulator.
  __device__ void flush(int64_t j0, int n) const {
    using A = Arith<Real>;
    Real e = Real(0), ex = Real(0), ey = Real(0), ez = Real(0);
    if (lane < n) observe(slot(j0 + lane), e, ex, ey, ez);
    const Real m2 = ex * ex + ey * ey + ez * ez;
    const Real m = sqrt(m2);
    for (int k = warp; k <= MP_R_MMZ; k += nwarps) {
      Real v;
      switch (k) {  // k is the same in every lane of the warp
        case MP_R_E: v = e; break;
        case MP_R_E2: v = e * e; break;
        case MP_R_M: v = m; break;
        case MP_R_M2: v = m2; break;
        case MP_R_M4: v = m2 * m2; break;
        case MP_R_MX: v = ex; break;
        case MP_R_MY: v = ey; break;
        case MP_R_MZ: v = ez; break;
        case MP_R_MZ2: v = ez * ez; break;
        case MP_R_AMZ: v = fabs(ez); break;
        case MP_R_EM: v = e * m; break;
        case MP_R_EMZ: v = e * ez; break;
        default: v = m * ez; break;  // MP_R_MMZ
      }
      if (lane >= n) v = Real(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        if (o < R) v += A::shfl(v, o);
      }
      if (lane == 0) acc[k] += static_cast<double>(v);
    }
  }
  // At measurement sweep j (the current one), after its first barrier: flush
  // the previous half.
  __device__ void maybe_flush(int64_t j) const {
    if ((cur == 0 || cur == R) && j > j_first) {
      const int64_t j0 = j - R > j_first ? j - R : j_first;
      flush(j0, static_cast<int>(j - j0));
    }
  }
  // After the call's last sweep and its barrier: flush the rest of the
  // measurement sweeps j_first .. n_meas-1 and keep the final state.
  __device__ void finish(int64_t n_meas) const {
    const int64_t last = n_meas - 1;
    if (last < j_first) return;  // no measurement sweep in this call
    int64_t j0 = last - last % R;
    if (j0 < j_first) j0 = j_first;
    flush(j0, static_cast<int>(last - j0) + 1);
    if (tid == 0) {  // the final state: the paper's per-path output
      Real e, ex, ey, ez;
      observe(slot(last), e, ex, ey, ez);
      acc[MP_R_FMX] = static_cast<double>(ex);
      acc[MP_R_FMY] = static_cast<double>(ey);
      acc[MP_R_FMZ] = static_cast<double>(ez);
      acc[MP_R_FE] = static_cast<double>(e);
    }
  }
  // Reduce the acceptance count and the worst | |S| - 1 | over the group and
  // write the path's record (the ring area is reused; call after a barrier).
  __device__ void write_record(double* rec, int accepted, double worst, int64_t nsweeps,
                               int64_t n_meas, int N, int tp, int bar, double accepted_before,
                               double* save_accepted) const {
    double nacc = static_cast<double>(accepted);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
      worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    }
    double* fin = reinterpret_cast<double*>(red);  // 2 doubles per warp
    if (lane == 0) {
      fin[2 * warp + 0] = nacc;
      fin[2 * warp + 1] = worst;
    }
    group_sync(tp, bar);
    if (tid == 0) {
      double tot = accepted_before, wmax = 0.0;
      for (int w = 0; w < nwarps; ++w) {
        tot += fin[2 * w + 0];
        wmax = fmax(wmax, fin[2 * w + 1]);
      }
      if (save_accepted) *save_accepted = tot;
      const double inv = n_meas > 0 ? 1.0 / static_cast<double>(n_meas) : NAN;
      for (int k = MP_R_E; k <= MP_R_MMZ; ++k) rec[k] = acc[k] * inv;
      for (int k = MP_R_FMX; k <= MP_R_FE; ++k) rec[k] = acc[k];
      rec[MP_R_ACC] = tot / (static_cast<double>(nsweeps) * static_cast<double>(N));
      rec[MP_R_NORM] = wmax;
      rec[MP_R_SPARE] = 0.0;
    }
  }
};

// Initial spin of site i: uniform on the sphere (Sec. 2.2), uniform angles,
// or the ordered start of Sec. 5.
template <typename Real>
__device__ __forceinline__ void initial_spin(uint32_t i, uint32_t c2, uint32_t c3i,
                                             const SweepParams& P, int mode, Real& x, Real& y,
                                             Real& z) {
  using A = Arith<Real>;
  const Philox4 r = philox4x32_10(i, 0u, c2, c3i, P.key);
  if (mode == MP_INIT_ORDERED) {
    x = Real(0);
    y = Real(0);
    z = Real(1);
  } else if (mode == MP_INIT_ANGLES) {
    A::init_angles(r.x, r.y, x, y, z);
  } else {
    A::trial(r.x, r.y, x, y, z);
  }
}

// --------------------------------------------------------- resumable state --
// A path's state in HBM (resumable runs): [acc: 24 doubles][accepted: double]
// padded to kStateHeader bytes, then its spins.
__device__ __forceinline__ unsigned char* path_state(const SweepParams& P, int sys_idx, int64_t path) {
  return P.state ? P.state + P.state_offset[sys_idx] + path * P.state_stride[sys_idx] : nullptr;
}

// Poll of the host's cancel flag by one thread of the group, every kCancelPoll
// sweeps of a call; the group reads the verdict after its next barrier.
__device__ __forceinline__ void poll_cancel(const SweepParams& P, int64_t s, int tid, int* flag) {
  if (tid == 0 && P.cancel != nullptr && ((s - P.s_begin) % kCancelPoll) == 0 && *P.cancel != 0) {
    *flag = 1;
    atomicExch(P.error, kErrCanceled);
  }
}

// ------------------------------------------------------------- one path --
// The lattice lives in the slice's shared memory, or in HBM at `hbm_spins`
// (the same layout) when it is updated in place there.
template <typename Real, class Geom>
__device__ __forceinline__ void run_path(const Geom geo, const DevSystem& sy, int sys_idx,
                                         int64_t path, const SweepParams& P, unsigned char* slice,
                                         int tid, int tp, int bar, Real* hbm_spins = nullptr) {
  using A = Arith<Real>;
  Real* sp = hbm_spins ? hbm_spins : reinterpret_cast<Real*>(slice + slice_spin_offset(tp, sy.ring));
  const int S = geo.stride();
  const uint32_t c2 = static_cast<uint32_t>(sy.path_begin + path);  // path id
  const uint32_t c3u = kTagUpdate | (static_cast<uint32_t>(sys_idx) << 8);
  const uint32_t c3i = kTagInit | (static_cast<uint32_t>(sys_idx) << 8);
  const int init = path_init_mode(P.init_mode, path, sy.n_paths);
  const Real J = static_cast<Real>(sy.J), hf = static_cast<Real>(sy.h);
  const Real bp = A::beta_param(sy.beta);
  // column segments per column (column_segments; 0 = decode every site: open
  // chains), and the host's table of the column-walk units when it was made
  // for this chunk (the table's K is then that of the same rule)
  int K = 0;
  const int4* units = nullptr;
  if constexpr (Geom::kColumns) {
    constexpr int LL = 2 * Geom::HL;
    constexpr int U = kColumnChunk<Real, Geom>;
    static_assert(LL % U == 0, "a whole column is a whole number of chunks");
    static_assert(Geom::HP * LL < 65536, "unit tables hold half indices in 16 bits");
    if (P.units != nullptr && sy.unit_off >= 0 && sy.unit_U == U && sy.unit_K > 0) {
      K = sy.unit_K;
      units = P.units + sy.unit_off;
    } else {
      K = column_segments(LL, U, tp);
    }
  }
  const int64_t j_first = P.s_begin > P.n_therm ? P.s_begin - P.n_therm : 0;
  Meter<Real> meter{reinterpret_cast<double*>(slice + slice_acc_offset()),
                    reinterpret_cast<Real*>(slice + slice_red_offset()),
                    sy.ring, tp >> 5, tid & 31, tid >> 5, tid,
                    1.0 / static_cast<double>(sy.N), J, hf, j_first};
  meter.start();
  unsigned char* st = path_state(P, sys_idx, path);
  Real* st_spins = st ? reinterpret_cast<Real*>(st + kStateHeader) : nullptr;
  __shared__ int cancel_flag[kMaxGroups];
  const int gidx = bar - 1;

  if (P.resume && st) {  // continue from the saved state
    for (int k = tid; k < 6 * S; k += tp) sp[k] = st_spins[k];
    if (tid < kAccDoubles) meter.acc[tid] = reinterpret_cast<const double*>(st)[tid];
  } else {
    for (int c = 0; c < 2; ++c) {
      const SpinView<Real> own(sp + c * 3 * S, S);
      const int cnt = geo.count(c);
      for (int hh = tid; hh < cnt; hh += tp) {
        int nb[Geom::NNB];
        int nn;
        const int i = geo.site(hh, c, nb, nn);
        Real x, y, z;
        initial_spin<Real>(static_cast<uint32_t>(i), c2, c3i, P, init, x, y, z);
        own.st(hh, x, y, z);
      }
    }
    if (tid < kAccDoubles) meter.acc[tid] = 0.0;
  }
  const double accepted_before =
      (P.resume && st) ? reinterpret_cast<const double*>(st)[kAccDoubles] : 0.0;
  if (tid == 0) cancel_flag[gidx] = 0;
  group_sync(tp, bar);

  int accepted = 0;
  bool canceled = false;
  for (int64_t s = P.s_begin; s < P.s_end; ++s) {
    const uint32_t sw = static_cast<uint32_t>(s);
    const PhiloxPrefix pre = philox_prefix(sw, c2, c3u, P.key);
    Partials<Real> part{Real(0), Real(0), Real(0), Real(0)};
    poll_cancel(P, s, tid, &cancel_flag[gidx]);
    if (s < P.n_therm) {
      half_sweep<Real, Geom, false, false>(geo, 0, pre, P.key, sp, tid, tp, K, units, J, hf,
                                           bp, accepted, part);
      group_sync(tp, bar);
      if (cancel_flag[gidx]) {
        canceled = true;
        break;
      }
      half_sweep<Real, Geom, false, false>(geo, 1, pre, P.key, sp, tid, tp, K, units, J, hf,
                                           bp, accepted, part);
      group_sync(tp, bar);
      continue;
    }
    // Measurement sweep j.  Colour-0 sites keep their values during the
    // colour-1 pass, so the colour-1 local fields give every bond once.
    const int64_t j = s - P.n_therm;
    half_sweep<Real, Geom, true, false>(geo, 0, pre, P.key, sp, tid, tp, K, units, J, hf, bp,
                                        accepted, part);
    group_sync(tp, bar);
    if (cancel_flag[gidx]) {
      canceled = true;
      break;
    }
    meter.maybe_flush(j);
    half_sweep<Real, Geom, true, true>(geo, 1, pre, P.key, sp, tid, tp, K, units, J, hf, bp,
                                       accepted, part);
    meter.record(part);
    group_sync(tp, bar);
  }
  if (canceled) {  // the call is discarded: no record, no saved state
    group_sync(tp, bar);
    return;
  }
  const int64_t n_meas_done = P.s_end > P.n_therm ? P.s_end - P.n_therm : 0;
  meter.finish(n_meas_done);
  group_sync(tp, bar);

  Real worst = Real(0);
  for (int c = 0; c < 2; ++c) {
    const SpinView<Real> own(sp + c * 3 * S, S);
    for (int hh = tid; hh < geo.count(c); hh += tp) {
      const V3<Real> v = own.ld(hh);
      worst = fmax(worst, fabs(sqrt(v.x * v.x + v.y * v.y + v.z * v.z) - Real(1)));
    }
  }
  if (P.save && st) {
    for (int k = tid; k < 6 * S; k += tp) st_spins[k] = sp[k];
    if (tid < kAccDoubles) reinterpret_cast<double*>(st)[tid] = meter.acc[tid];
  }
  meter.write_record(P.records + (sy.rec_offset + path) * MP_NREC, accepted,
                     static_cast<double>(worst), P.s_end, n_meas_done, sy.N, tp, bar,
                     accepted_before, (P.save && st) ? reinterpret_cast<double*>(st) + kAccDoubles : nullptr);
  if (P.spins != nullptr) {
    double* out = P.spins + P.spin_offset[sys_idx] + path * 3 * static_cast<int64_t>(sy.N);
    for (int c = 0; c < 2; ++c) {
      const SpinView<Real> own(sp + c * 3 * S, S);
      for (int hh = tid; hh < geo.count(c); hh += tp) {
        int nb[Geom::NNB];
        int nn;
        const int i = geo.site(hh, c, nb, nn);
        const V3<Real> v = own.ld(hh);
        out[3 * i + 0] = v.x;
        out[3 * i + 1] = v.y;
        out[3 * i + 2] = v.z;
      }
    }
  }
  group_sync(tp, bar);  // the slice is reused by the next item
}

// ------------------------------------------------ two-CTA clusters -------
// A simple cubic lattice too large for one SM's shared memory but not for
// two (FP32 L = 32: 393 KB of spins) is held by the two CTAs of a cluster:
// CTA rank r keeps the z-planes r L/2 .. r L/2 + L/2 - 1, and in each colour
// array also one halo plane on either side (local planes 0 and L/2 + 1) with
// the partner's boundary plane.  A half-sweep of colour c updates the local
// planes by the same column walk as run_path (the halo planes give the +-z
// neighbours across the cut, so no index wraps in z), and each thread pushes
// the new values of its column's two boundary sites straight into the
// partner's halo planes of colour c (distributed shared memory stores).  The
// partner reads colour c only in the next half-sweep, after the cluster
// barrier that ends this one, so one barrier per half-sweep orders
// everything; during a half-sweep each CTA reads only colour 1 - c and writes
// only colour c.  Measurement partials of the partner's warps go into the
// owner's (rank 0's) partial-sum ring, which then holds every warp of the
// lattice; rank 0 flushes, keeps the FP64 accumulators and writes the record.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}
// Generic address of the same shared-memory location in CTA `rank` of the cluster.
template <typename T>
__device__ __forceinline__ T* map_rank(T* p, uint32_t rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
  return reinterpret_cast<T*>(out);
}
// Every thread of both CTAs; release/acquire at cluster scope, so shared
// memory written (locally or remotely) before it is visible after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

template <int L>
struct PairGeom {
  static constexpr int HL = L / 2, HP = L * L / 2;
  static constexpr int ZL = L / 2;       // planes per CTA
  static constexpr int S = HP * (ZL + 2);  // sites per colour array, with the two halo planes
  static_assert(6 * S * 4 == pair_spin_bytes(L, 4), "pair layout");
};

// Planes of a column walked per unrolled chunk (even, so that each site's x
// parity is fixed at compile time): 8, 0.4% faster than 4 on the batch of
// uneven sizes.
constexpr int kPairChunk = 8;

template <typename Real, int L, bool kMeas, bool kEnergy>
__device__ __forceinline__ void half_sweep_pair(int c, int zbase, const PhiloxPrefix& pre,
                                                const PhiloxKeys& key, Real* sp, Real* partner_sp,
                                                int tid, int tp, Real J, Real hf, Real bp,
                                                int& accepted, Partials<Real>& part) {
  using G = PairGeom<L>;
  constexpr int HL = G::HL, HP = G::HP, ZL = G::ZL, S = G::S;
  const SpinView<Real> own(sp + c * 3 * S, S), oth(sp + (1 - c) * 3 * S, S);
  const SpinView<Real> halo(partner_sp + c * 3 * S, S);  // the partner's array of colour c
  for (int col = tid; col < HP; col += tp) {
    const int hx = col % HL;
    const int y = col / HL;
    const int oyp = (y == L - 1) ? -(L - 1) * HL : HL;
    const int oym = (y == 0) ? (L - 1) * HL : -HL;
    const int oxp1 = (hx == HL - 1) ? -(HL - 1) : 1;  // +x offset when x is odd
    const int oxm0 = (hx == 0) ? (HL - 1) : -1;         // -x offset when x is even
    // x parity of the sites in local planes 1, 3, ... (pa) and 2, 4, ... (pb):
    // chunks have an even number of planes, so within one the choice of
    // parity and x-neighbour offset is made at compile time
    const int pa = (y + zbase + c) & 1, pb = pa ^ 1;
    const int oxa = pa ? oxp1 : oxm0, oxb = pa ? oxm0 : oxp1;
    int hh = col + HP;                                   // local plane 1
    V3<Real> o0 = oth.ld(hh);       // the other colour at the site's half index
    V3<Real> mz = oth.ld(hh - HP);  // -z neighbour (halo plane 0)
    static_assert(kPairChunk % 2 == 0 && ZL % kPairChunk == 0, "even chunks that tile the planes");
    for (int zc = 0; zc < ZL; zc += kPairChunk) {
#pragma unroll
      for (int k = 0; k < kPairChunk; ++k, hh += HP) {
        // global plane zbase + zc + k
        const int p = (k & 1) ? pb : pa;
        const int nxo = hh + ((k & 1) ? oxb : oxa);
        const V3<Real> cz = oth.ld(hh + HP);
        const V3<Real> f =
            add3(add3(add3(add3(add3(o0, oth.ld(nxo)), oth.ld(hh + oyp)), oth.ld(hh + oym)), cz), mz);
        // site index x + L(y + L z_global) = 2 (col + HP z_global) + p
        update<Real, kMeas, kEnergy>(static_cast<uint32_t>(2 * (hh + HP * (zbase - 1)) + p), pre, key,
                                     own, hh, f.x, f.y, f.z, J, hf, bp, accepted, part);
        mz = o0;
        o0 = cz;
      }
    }
    // the column's boundary sites to the partner's halo planes: local plane 1
    // is the partner's plane ZL + 1, local plane ZL its plane 0
    const V3<Real> a = own.ld(col + HP);
    halo.st(col + HP * (ZL + 1), a.x, a.y, a.z);
    const V3<Real> b = own.ld(col + HP * ZL);
    halo.st(col, b.x, b.y, b.z);
  }
}

// One path of a simple cubic L (= kPairL) lattice on the two CTAs of a
// cluster; every thread of both CTAs calls it with the same arguments except
// `rank` and tid.  The record, the saved accumulators and the acceptance
// count are written by rank 0; each rank saves and outputs its own planes.
template <typename Real, int L>
__device__ void run_path_pair(const DevSystem& sy, int sys_idx, int64_t path, const SweepParams& P,
                              unsigned char* slice, int tid, int tp, uint32_t rank) {
  using A = Arith<Real>;
  using G = PairGeom<L>;
  constexpr int HL = G::HL, HP = G::HP, ZL = G::ZL, S = G::S;
  constexpr int NH = L * L * L / 2;  // sites per colour of the whole lattice
  // rank 0's ring holds the partials of both CTAs' warps
  Real* sp = reinterpret_cast<Real*>(slice + slice_spin_offset(2 * tp, sy.ring));
  Real* partner_sp = map_rank(sp, rank ^ 1u);
  const int zbase = static_cast<int>(rank) * ZL;
  const uint32_t c2 = static_cast<uint32_t>(sy.path_begin + path);  // path id
  const uint32_t c3u = kTagUpdate | (static_cast<uint32_t>(sys_idx) << 8);
  const uint32_t c3i = kTagInit | (static_cast<uint32_t>(sys_idx) << 8);
  const int init = path_init_mode(P.init_mode, path, sy.n_paths);
  const Real J = static_cast<Real>(sy.J), hf = static_cast<Real>(sy.h);
  const Real bp = A::beta_param(sy.beta);
  const int64_t j_first = P.s_begin > P.n_therm ? P.s_begin - P.n_therm : 0;
  Real* red0 = reinterpret_cast<Real*>(slice + slice_red_offset());
  Meter<Real> meter{reinterpret_cast<double*>(slice + slice_acc_offset()),
                    rank == 0 ? red0 : map_rank(red0, 0u),
                    sy.ring, tp >> 5, tid & 31, tid >> 5, tid,
                    1.0 / static_cast<double>(sy.N), J, hf, j_first};
  meter.nslot = 2 * (tp >> 5);
  meter.slot_off = rank == 0 ? 0 : (tp >> 5);
  meter.start();
  unsigned char* st = path_state(P, sys_idx, path);
  Real* st_spins = st ? reinterpret_cast<Real*>(st + kStateHeader) : nullptr;
  __shared__ int pair_cancel;
  __shared__ double pair_xch[2];  // rank 1's acceptance count and worst | |S| - 1 |, on rank 0
  const bool resume = P.resume && st;

  // local plane zl holds global plane (zbase + zl - 1) mod L, zl = 0 .. ZL + 1
  for (int c = 0; c < 2; ++c) {
    const SpinView<Real> own(sp + c * 3 * S, S);
    for (int h = tid; h < S; h += tp) {
      const int col = h % HP, zl = h / HP;
      const int zg = (zbase + zl - 1 + L) % L;
      const int hg = col + HP * zg;  // half index in the whole lattice
      Real x, y, z;
      if (resume) {
        const SpinView<Real> saved(st_spins + c * 3 * NH, NH);
        const V3<Real> v = saved.ld(hg);
        x = v.x;
        y = v.y;
        z = v.z;
      } else {
        const int p = (col / HL + zg + c) & 1;
        initial_spin<Real>(static_cast<uint32_t>(2 * hg + p), c2, c3i, P, init, x, y, z);
      }
      own.st(h, x, y, z);
    }
  }
  if (tid < kAccDoubles) meter.acc[tid] = (resume && rank == 0) ? reinterpret_cast<const double*>(st)[tid] : 0.0;
  const double accepted_before = (resume && rank == 0) ? reinterpret_cast<const double*>(st)[kAccDoubles] : 0.0;
  if (tid == 0) pair_cancel = 0;
  cluster_sync_all();

  int accepted = 0;
  bool canceled = false;
  for (int64_t s = P.s_begin; s < P.s_end; ++s) {
    const uint32_t sw = static_cast<uint32_t>(s);
    const PhiloxPrefix pre = philox_prefix(sw, c2, c3u, P.key);
    Partials<Real> part{Real(0), Real(0), Real(0), Real(0)};
    // rank 0 polls the host's flag and tells both CTAs, so that they stop together
    if (rank == 0 && tid == 0 && P.cancel != nullptr && ((s - P.s_begin) % kCancelPoll) == 0 &&
        *P.cancel != 0) {
      pair_cancel = 1;
      *map_rank(&pair_cancel, 1u) = 1;
      atomicExch(P.error, kErrCanceled);
    }
    const bool meas = s >= P.n_therm;
    if (meas)
      half_sweep_pair<Real, L, true, false>(0, zbase, pre, P.key, sp, partner_sp, tid, tp, J, hf, bp,
                                            accepted, part);
    else
      half_sweep_pair<Real, L, false, false>(0, zbase, pre, P.key, sp, partner_sp, tid, tp, J, hf, bp,
                                             accepted, part);
    cluster_sync_all();
    if (pair_cancel) {
      canceled = true;
      break;
    }
    if (meas) {
      if (rank == 0) meter.maybe_flush(s - P.n_therm);
      half_sweep_pair<Real, L, true, true>(1, zbase, pre, P.key, sp, partner_sp, tid, tp, J, hf, bp,
                                           accepted, part);
      meter.record(part);
    } else {
      half_sweep_pair<Real, L, false, false>(1, zbase, pre, P.key, sp, partner_sp, tid, tp, J, hf, bp,
                                             accepted, part);
    }
    cluster_sync_all();
  }
  if (canceled) {  // the call is discarded: no record, no saved state
    cluster_sync_all();
    return;
  }
  const int64_t n_meas_done = P.s_end > P.n_therm ? P.s_end - P.n_therm : 0;
  if (rank == 0) meter.finish(n_meas_done);
  __syncthreads();  // the ring area is free from here on (finish has read its last slot)

  // this CTA's planes: worst | |S| - 1 |, saved state, final spins
  Real worst = Real(0);
  for (int c = 0; c < 2; ++c) {
    const SpinView<Real> own(sp + c * 3 * S, S);
    for (int h = tid + HP; h < HP * (ZL + 1); h += tp) {
      const V3<Real> v = own.ld(h);
      worst = fmax(worst, fabs(sqrt(v.x * v.x + v.y * v.y + v.z * v.z) - Real(1)));
      const int col = h % HP, zg = zbase + h / HP - 1;
      const int hg = col + HP * zg;
      if (P.save && st) SpinView<Real>(st_spins + c * 3 * NH, NH).st(hg, v.x, v.y, v.z);
      if (P.spins != nullptr) {
        const int i = 2 * hg + ((col / HL + zg + c) & 1);
        double* out = P.spins + P.spin_offset[sys_idx] + path * 3 * static_cast<int64_t>(sy.N) + 3 * i;
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
      }
    }
  }
  // acceptance count and worst norm of this CTA; rank 1 hands its totals to rank 0
  double nacc = static_cast<double>(accepted), wst = static_cast<double>(worst);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
    wst = fmax(wst, __shfl_xor_sync(0xffffffffu, wst, o));
  }
  double* pair_red = reinterpret_cast<double*>(red0);  // this CTA's own ring area
  if ((tid & 31) == 0) {
    pair_red[2 * (tid >> 5)] = nacc;
    pair_red[2 * (tid >> 5) + 1] = wst;
  }
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0, wmax = 0.0;
    for (int w = 0; w < (tp >> 5); ++w) {
      tot += pair_red[2 * w];
      wmax = fmax(wmax, pair_red[2 * w + 1]);
    }
    if (rank == 1) {
      double* x = map_rank(pair_xch, 0u);
      x[0] = tot;
      x[1] = wmax;
    } else {
      pair_red[0] = tot;
      pair_red[1] = wmax;
    }
  }
  cluster_sync_all();  // rank 1's totals are in rank 0's pair_xch
  if (rank == 0 && tid == 0) {
    const double tot = accepted_before + pair_red[0] + pair_xch[0];
    const double wmax = fmax(pair_red[1], pair_xch[1]);
    double* rec = P.records + (sy.rec_offset + path) * MP_NREC;
    const double inv = n_meas_done > 0 ? 1.0 / static_cast<double>(n_meas_done) : NAN;
    for (int k = MP_R_E; k <= MP_R_MMZ; ++k) rec[k] = meter.acc[k] * inv;
    for (int k = MP_R_FMX; k <= MP_R_FE; ++k) rec[k] = meter.acc[k];
    rec[MP_R_ACC] = tot / (static_cast<double>(P.s_end) * static_cast<double>(sy.N));
    rec[MP_R_NORM] = wmax;
    rec[MP_R_SPARE] = 0.0;
    if (P.save && st) {
      for (int k = 0; k < kAccDoubles; ++k) reinterpret_cast<double*>(st)[k] = meter.acc[k];
      reinterpret_cast<double*>(st)[kAccDoubles] = tot;
    }
  }
  cluster_sync_all();  // the slices (and pair_xch) are reused by the next item
}

// ------------------------------------------------------ TMA primitives --
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// End an mbarrier's life before its memory is initialised again or reused.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing on the mbarrier `bar`.
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bulk copy shared -> global, as its own bulk group.
__device__ __forceinline__ void tma_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until at most N (a constant) bulk store groups may still read shared memory.
template <int N>
__device__ __forceinline__ void tma_wait_read_n() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
#define tma_wait_read(n) tma_wait_read_n<n>()
__device__ __forceinline__ void tma_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the mbarrier, giving up after about 2 s: then the
// error flag is set and false returned (the caller stops the path cleanly).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* error) {
  const uint32_t a = smem_addr(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 0) {
      const uint64_t t = global_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > 2000000000ull) {
        atomicExch(error, 1);
        return false;
      }
    }
  }
}

// ---------------------------------------------------- streamed from HBM --
// Lattices too large for shared memory.  Each path's spins stay in HBM in the
// layout [z][colour][(x, y) pairs | z][L*L/2] (a "half-plane" is one colour
// of one z-plane, padded to 16 bytes), in a buffer owned by the thread group for the
// whole run.  A sweep walks the z-planes as a wavefront over a ring of 4 + 5
// half-plane buffers in shared memory, filled by TMA bulk copies and written
// back by bulk stores:
//   step q = 0 .. L+1:  (a) colour-0 update of plane q          (q < L)
//                       (b) colour-1 update of plane (q-1) mod L (q >= 2)
// Colour 0 of plane q needs colour 1 of planes q-1, q, q+1 still old; colour 1
// of plane q-1 needs colour 0 of planes q-2, q-1, q already new; plane 0's
// colour-1 update waits until the end (it needs colour 0 of plane L-1 new,
// and colour 0 of plane L-1 needs colour 1 of plane 0 old).  Every update thus
// sees exactly the neighbour values of the two-pass checkerboard sweep.
// Phases (a) and (b) of a step run back to back, with one group barrier per
// step (see the loop below for why no barrier is needed between them).
// Ring indices: colour-0 step index q' = 0..L+1 (planes 0..L-1, 0, 1) in slot
// q' mod 4; colour-1 step index q' = -1..L (planes L-1, 0..L-1, 0) in slot
// (q'+1) mod 5.  Every load is issued two steps before its first use.
constexpr int kSlots = 9;  // half-plane buffers per streamed path: 4 for colour 0, 5 for colour 1

template <typename Real>
struct StreamLayout {
  static __host__ __device__ int hps(int L) {  // padded half-plane, in Reals
    const int bytes = (3 * (L * L / 2) * static_cast<int>(sizeof(Real)) + 15) / 16 * 16;
    return bytes / static_cast<int>(sizeof(Real));
  }
};

// kL > 0: the lattice size is the compile-time constant kL, which turns the
// in-plane index arithmetic and the buffer offsets into immediates; kL = 0:
// any even L (sy.L).  kRS > 0: tp = kRS * L/2 threads per path, so every
// thread owns exactly kL / kRS rows at compile-time offsets.
template <typename Real, int kL, int kRS>
__device__ void run_path_streamed(const DevSystem& sy, int sys_idx, int64_t path,
                                  const SweepParams& P, unsigned char* slice, int tid, int tp,
                                  int bar, Real* lat_cta) {
  using A = Arith<Real>;
  const int L = kL > 0 ? kL : sy.L, HL = L / 2, HP = L * L / 2;
  const int hps = StreamLayout<Real>::hps(L);
  const uint32_t bytes = static_cast<uint32_t>(hps * sizeof(Real));
  // [9 mbarriers][9 load counters] in 128 bytes, then the 9 half-plane buffers
  uint64_t* mbar = reinterpret_cast<uint64_t*>(slice + slice_spin_offset(tp, sy.ring));
  uint32_t* issued = reinterpret_cast<uint32_t*>(mbar + kSlots);
  Real* buf = reinterpret_cast<Real*>(slice + slice_spin_offset(tp, sy.ring) + 128);
  // buffer of colour c, step index q (see above): 4 slots for colour 0, 5 for colour 1
  auto c0buf = [&](int q) { return buf + (q & 3) * hps; };
  auto c1buf = [&](int q) { return buf + (4 + (q + 1) % 5) * hps; };
  auto c0bar = [&](int q) { return mbar + (q & 3); };
  auto c1bar = [&](int q) { return mbar + 4 + (q + 1) % 5; };
  // a resumable run keeps the path's lattice in its state; otherwise the
  // group's own HBM buffer holds it for the run
  unsigned char* st = path_state(P, sys_idx, path);
  Real* lat = st ? reinterpret_cast<Real*>(st + kStateHeader) : lat_cta;
  auto plane = [&](int z, int c) { return lat + (static_cast<int64_t>(z) * 2 + c) * hps; };
  auto wrap = [&](int q) { return ((q % L) + L) % L; };
  const uint32_t c2 = static_cast<uint32_t>(sy.path_begin + path);  // path id
  const uint32_t c3u = kTagUpdate | (static_cast<uint32_t>(sys_idx) << 8);
  const uint32_t c3i = kTagInit | (static_cast<uint32_t>(sys_idx) << 8);
  const int init = path_init_mode(P.init_mode, path, sy.n_paths);
  const Real J = static_cast<Real>(sy.J), hf = static_cast<Real>(sy.h);
  const Real bp = A::beta_param(sy.beta);
  const int64_t j_first = P.s_begin > P.n_therm ? P.s_begin - P.n_therm : 0;
  Meter<Real> meter{reinterpret_cast<double*>(slice + slice_acc_offset()),
                    reinterpret_cast<Real*>(slice + slice_red_offset()),
                    sy.ring, tp >> 5, tid & 31, tid >> 5, tid,
                    1.0 / static_cast<double>(sy.N), J, hf, j_first};
  meter.start();
  __shared__ int abort_flag[kMaxGroups];  // per thread group: a bounded wait gave up, or canceled
  const int gidx = bar - 1;
  const bool producer = tid == 0;
  const bool resume = P.resume && st;
  const double accepted_before = resume ? reinterpret_cast<const double*>(st)[kAccDoubles] : 0.0;

  // Initial state straight into HBM (generic stores), visible to the bulk copies.
  const int N = sy.N;
  for (int i = resume ? N : tid; i < N; i += tp) {
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    const int c = (x + y + z) & 1;
    Real sx, sy_, sz;
    initial_spin<Real>(static_cast<uint32_t>(i), c2, c3i, P, init, sx, sy_, sz);
    Real* hpl = plane(z, c);
    const int hp = (x >> 1) + HL * y;
    SpinView<Real>(hpl, HP).st(hp, sx, sy_, sz);
  }
  fence_async_global();
  if (tid < kAccDoubles) meter.acc[tid] = resume ? reinterpret_cast<const double*>(st)[tid] : 0.0;
  if (tid == 0) abort_flag[gidx] = 0;
  if (producer) {
    for (int k = 0; k < kSlots; ++k) {
      mbar_init(mbar + k, 1);
      issued[k] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  auto load = [&](Real* dst, const Real* src, int slot) {  // producer only
    ++issued[slot];
    tma_load(dst, src, bytes, mbar + slot);
  };
  group_sync(tp, bar);

  // In-plane thread layout: column hx, rows y0, y0 + RS, ...
  const int RS = kRS > 0 ? kRS : tp / HL;
  constexpr bool kFixedRows = kL > 0 && kRS > 0 && kL % kRS == 0;
  const bool active = tid < HL * RS;
  const int hx = active ? tid % HL : 0;
  const int y0 = active ? tid / HL : L;
  // loads per sweep into each ring slot, for the mbarrier phase parity: slot
  // j of a ring of n slots takes the shifted step indices j, j + n, ... <= L+1
  auto per_sweep = [&](int j, int n) { return (L + 1 - j) / n + 1; };
  int accepted = 0;
  bool ok = true;

  for (int64_t s = P.s_begin; s < P.s_end && ok; ++s) {
    const uint32_t sw = static_cast<uint32_t>(s);
    const PhiloxPrefix pre = philox_prefix(sw, c2, c3u, P.key);
    const bool meas = s >= P.n_therm;
    const int64_t j = s - P.n_therm;
    Partials<Real> part{Real(0), Real(0), Real(0), Real(0)};
    const int64_t sc = s - P.s_begin;  // sweeps since the mbarriers were initialised
    auto parity0 = [&](int q) {
      return static_cast<uint32_t>((sc * per_sweep(q & 3, 4) + q / 4) & 1);
    };
    auto parity1 = [&](int q) {
      const int qq = q + 1;
      return static_cast<uint32_t>((sc * per_sweep(qq % 5, 5) + qq / 5) & 1);
    };
    // Buffers first used at step q: colour-0 index q, colour-1 index q+1 (at
    // q = 0 also colour-1 indices -1 and 0).  Only the producer waits on their
    // mbarriers; the group barrier after the wait hands the data to everyone.
    auto wait_step = [&](int q) {
      bool w = mbar_wait(c0bar(q), parity0(q), P.error);
      if (q == 0) {
        w = w && mbar_wait(c1bar(-1), parity1(-1), P.error);
        w = w && mbar_wait(c1bar(0), parity1(0), P.error);
      }
      if (q < L) w = w && mbar_wait(c1bar(q + 1), parity1(q + 1), P.error);
      if (!w) abort_flag[gidx] = 1;
    };
    int cancel = 0;
    poll_cancel(P, s, tid, &cancel);
    if (producer && cancel) abort_flag[gidx] = 1;  // stop before any copy of this sweep
    if (producer && !cancel) {
      tma_wait_all();  // the previous sweep's write-backs are complete
      if (!(P.test_stall && s == P.s_begin)) load(c0buf(0), plane(0, 0), 0);
      load(c0buf(1), plane(1 % L, 0), 1);
      for (int q1 = -1; q1 <= 2; ++q1) load(c1buf(q1), plane(wrap(q1), 1), 4 + (q1 + 1) % 5);
      wait_step(0);
    }
    group_sync(tp, bar);
    if (abort_flag[gidx]) {
      ok = false;
      break;
    }
    // One colour phase over plane z: own, same-plane, +z and -z buffers.  The
    // thread's column hx is fixed, so its +-x offsets for either parity of x
    // are too (oxp1: +x when x is odd, oxm0: -x when x is even).
    const int oxp1 = (hx == HL - 1) ? -(HL - 1) : 1;
    const int oxm0 = (hx == 0) ? (HL - 1) : -1;
    auto phase = [&](int c, int z, Real* own_base, Real* same_base, Real* up_base, Real* dn_base,
                     bool energy) {
      const SpinView<Real> own(own_base, HP), same(same_base, HP), up(up_base, HP), dn(dn_base, HP);
      auto row = [&](int y) {
        const int hp = hx + HL * y;
        const int p = (y + z + c) & 1;
        const int xp = hp + (p ? oxp1 : 0);
        const int xm = hp + (p ? 0 : oxm0);
        const int yp = (y == L - 1) ? hp - (L - 1) * HL : hp + HL;
        const int ym = (y == 0) ? hp + (L - 1) * HL : hp - HL;
        const V3<Real> f = add3(add3(add3(add3(add3(same.ld(xp), same.ld(xm)), same.ld(yp)), same.ld(ym)),
                                     up.ld(hp)), dn.ld(hp));
        const uint32_t i = static_cast<uint32_t>(2 * (hp + HP * z) + p);
        if (meas) {
          if (energy)
            update<Real, true, true>(i, pre, P.key, own, hp, f.x, f.y, f.z, J, hf, bp,
                                     accepted, part);
          else
            update<Real, true, false>(i, pre, P.key, own, hp, f.x, f.y, f.z, J, hf, bp,
                                      accepted, part);
        } else {
          update<Real, false, false>(i, pre, P.key, own, hp, f.x, f.y, f.z, J, hf, bp,
                                     accepted, part);
        }
      };
      if constexpr (kFixedRows) {
        if (active) {
          // Rows y0 + k kRS: the x parity of row k is that of row 0 flipped
          // when k kRS is odd, and only the first row can be row 0 and only
          // the last row L - 1, so parity, x offset and the y wraps are fixed
          // at compile time for all but those.
          constexpr int kRows = kL / kRS;
          const int pz = (y0 + z + c) & 1;
          const int xoa = pz ? oxp1 : oxm0, xob = pz ? oxm0 : oxp1;
#pragma unroll
          for (int k = 0; k < kRows; ++k) {
            const int y = y0 + k * kRS;
            const bool flip = ((k * kRS) & 1) != 0;
            const int p = flip ? pz ^ 1 : pz;
            const int hp = hx + HL * y;
            const int xo = hp + (flip ? xob : xoa);
            const int yp = (k == kRows - 1 && y == L - 1) ? hp - (L - 1) * HL : hp + HL;
            const int ym = (k == 0 && y == 0) ? hp + (L - 1) * HL : hp - HL;
            // the two x neighbours in either order (a + b = b + a exactly)
            const V3<Real> f = add3(add3(add3(add3(add3(same.ld(hp), same.ld(xo)), same.ld(yp)), same.ld(ym)),
                                         up.ld(hp)), dn.ld(hp));
            const uint32_t i = static_cast<uint32_t>(2 * (hp + HP * z) + p);
            if (meas) {
              if (energy)
                update<Real, true, true>(i, pre, P.key, own, hp, f.x, f.y, f.z, J, hf, bp, accepted, part);
              else
                update<Real, true, false>(i, pre, P.key, own, hp, f.x, f.y, f.z, J, hf, bp, accepted, part);
            } else {
              update<Real, false, false>(i, pre, P.key, own, hp, f.x, f.y, f.z, J, hf, bp, accepted, part);
            }
          }
        }
      } else {
#pragma unroll 4
        for (int y = y0; y < L; y += RS) row(y);
      }
    };
    // One barrier per step.  A thread updates the same half indices hp in
    // both phases, and the colour-1 site at (hp, plane q-1) has the colour-0
    // site at (hp, plane q) as its +z neighbour: phase (b) reads the thread's
    // own results of phase (a), and every other value either phase reads was
    // written before the previous barrier (in-plane neighbours of the other
    // colour come from the previous step) or is written after the next one.
    for (int q = 0; q <= L + 1; ++q) {
      if (q < L) phase(0, q, c0buf(q), c1buf(q), c1buf(q + 1), c1buf(q - 1), false);
      if (q >= 2) phase(1, wrap(q - 1), c1buf(q - 1), c0buf(q - 1), c0buf(q), c0buf(q - 2), meas);
      fence_async_shared();
      // the buffers step q+1 starts with were issued at step q-1: the producer
      // confirms them now, and the barrier below hands them to every thread
      if (producer && q + 1 <= L + 1) wait_step(q + 1);
      group_sync(tp, bar);
      if (abort_flag[gidx]) {
        ok = false;
        break;
      }
      if (meas && q == 0) meter.maybe_flush(j);
      if (producer) {  // after the barrier: the buffers just written are complete
        if (q < L) tma_store(plane(q, 0), c0buf(q), bytes);
        if (q >= 2) tma_store(plane(wrap(q - 1), 1), c1buf(q - 1), bytes);
        // the slots refilled now last held colour-0 index q-2 (stored after
        // step q-2) and colour-1 index q-2 (stored after step q-1): all but
        // this step's (at most two) store groups must have finished reading
        // shared memory
        tma_wait_read(2);
        // colour-0 step indices L and L+1 reload planes 0 and 1 written this sweep
        if (q + 2 >= L) tma_wait_all();
        if (q + 2 <= L + 1) load(c0buf(q + 2), plane(wrap(q + 2), 0), (q + 2) & 3);
        if (q + 3 <= L) load(c1buf(q + 3), plane(wrap(q + 3), 1), 4 + (q + 4) % 5);
      }
    }
    if (!ok) break;
    if (meas) {
      meter.record(part);
      group_sync(tp, bar);
    }
  }
  if (producer) {
    if (!ok) {
      // a load did not arrive in time: wait (bounded) for every load still
      // in flight before the shared memory is given up
      for (int k = 0; k < kSlots; ++k)
        if (issued[k] > 0) mbar_wait(mbar + k, (issued[k] - 1) & 1, P.error);
    }
    tma_wait_all();
    fence_async_global();
    // every consumer passed its last wait before the last barrier
    for (int k = 0; k < kSlots; ++k) mbar_inval(mbar + k);
  }
  group_sync(tp, bar);
  if (!ok) return;  // the error flag is set; the path's record is not written
  const int64_t n_meas_done = P.s_end > P.n_therm ? P.s_end - P.n_therm : 0;
  meter.finish(n_meas_done);
  group_sync(tp, bar);

  Real worst = Real(0);  // in the working precision: FP64 runs at 1/64 rate on this GPU
  for (int i = tid; i < N; i += tp) {
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    const int hp = (x >> 1) + HL * y;
    const V3<Real> v = SpinView<Real>(plane(z, (x + y + z) & 1), HP).ld(hp);
    const Real a = v.x, b = v.y, c = v.z;
    worst = fmax(worst, fabs(sqrt(a * a + b * b + c * c) - Real(1)));
    if (P.spins != nullptr) {
      double* out = P.spins + P.spin_offset[sys_idx] + path * 3 * static_cast<int64_t>(N);
      out[3 * i + 0] = a;
      out[3 * i + 1] = b;
      out[3 * i + 2] = c;
    }
  }
  if (P.save && st && tid < kAccDoubles) reinterpret_cast<double*>(st)[tid] = meter.acc[tid];
  meter.write_record(P.records + (sy.rec_offset + path) * MP_NREC, accepted,
                     static_cast<double>(worst), P.s_end, n_meas_done, N, tp, bar, accepted_before,
                     (P.save && st) ? reinterpret_cast<double*>(st) + kAccDoubles : nullptr);
  group_sync(tp, bar);  // the slice and the HBM buffer are reused by the next item
}

// ------------------------------------------------------- persistent loop --
// The compile-time lattice sizes each precision supports in shared memory.
#define MPK_FOR_EACH_L_FP32(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26)
#define MPK_FOR_EACH_L_FP64(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20)

// Kernel variants: kLattice > 0 runs only simple cubic L = kLattice (a batch of
// one size), kLattice = kChainKernel only open chains, kLattice = kMixedKernel
// switches on each work item's lattice (a batch of uneven sizes).
constexpr int kMixedKernel = 0;
constexpr int kChainKernel = -1;
constexpr int kStreamKernel = -2;  // simple cubic lattices streamed from HBM (any even L)
// simple cubic lattices of one size L streamed from HBM, compiled for that L
__host__ __device__ constexpr int stream_variant(int L) { return -1000 - L; }
__host__ __device__ constexpr int stream_variant_L(int v) { return v <= -1000 ? -1000 - v : 0; }

template <typename Real, int kLattice>
__device__ __forceinline__ void dispatch_path(const DevSystem& sy, int sys_idx, int64_t path,
                                              const SweepParams& P, unsigned char* slice, int tid,
                                              int tp, int bar);

// Largest CTA of every sweep kernel: 512 threads with up to 128 registers per
// thread, which the FP64 form needs and which buys the FP32 column walk its
// unrolled instruction-level parallelism.  (1024-thread CTAs at 64 registers
// were measured 6-16% slower for L = 18 and 24.)
template <typename Real, int kLattice>
struct CtaLimit {
  static constexpr int value = 512;
};

template <typename Real, int kLattice>
__global__ void __launch_bounds__(CtaLimit<Real, kLattice>::value, 1)
    sweep_kernel(const SweepParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_item;
  if constexpr (kLattice == kMixedKernel && sizeof(Real) == 4) {
    // First the lattices held by two CTAs: the cluster takes one path at a
    // time from its own queue (rank 0 draws, both CTAs read), then each CTA
    // goes on to the single-CTA items below.
    if (P.n_pair_items > 0) {
      if (cluster_size() != 2) {
        if (threadIdx.x == 0) atomicExch(P.error, kErrLaunch);
      } else {
        __shared__ int s_pair;
        const uint32_t rank = cluster_rank();
        for (;;) {
          if (rank == 0 && threadIdx.x == 0) {
            const int it = atomicAdd(P.pair_queue, 1);
            s_pair = it;
            *map_rank(&s_pair, 1u) = it;
          }
          cluster_sync_all();
          const int item = s_pair;
          cluster_sync_all();  // both CTAs have read the item before rank 0 draws again
          if (item >= P.n_pair_items) break;
          const WorkItem it = P.pair_items[item];
          run_path_pair<Real, kPairL>(P.systems[it.sys], it.sys, it.path0, P, smem,
                                      static_cast<int>(threadIdx.x), static_cast<int>(blockDim.x), rank);
        }
      }
    }
  }
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
      bool done = false;
      if constexpr (stream_variant_L(kLattice) > 0) {
        Real* lat = reinterpret_cast<Real*>(
            static_cast<unsigned char*>(P.lattice) +
            (static_cast<int64_t>(blockIdx.x) * P.lattice_groups + g) * P.lattice_stride);
        constexpr int kL = stream_variant_L(kLattice);
        if (sy.tp == 8 * kL)  // 16 row groups of L/2 threads: L/16 rows per thread
          run_path_streamed<Real, kL, 16>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes,
                                          tid, sy.tp, 1 + g, lat);
        else if (sy.tp == 4 * kL)  // 8 row groups: L/8 rows per thread
          run_path_streamed<Real, kL, 8>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes,
                                         tid, sy.tp, 1 + g, lat);
        else
          run_path_streamed<Real, kL, 0>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes,
                                         tid, sy.tp, 1 + g, lat);
        done = true;
      }
      if constexpr (kLattice == kStreamKernel || kLattice == kMixedKernel || kLattice == kGlobalKernel) {
        if (!done && sy.mode == kModeGlobal) {
          Real* lat = reinterpret_cast<Real*>(
              static_cast<unsigned char*>(P.lattice) +
              (static_cast<int64_t>(blockIdx.x) * P.lattice_groups + g) * P.lattice_stride);
          run_path<Real>(GeomSCDyn{sy.L}, sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes, tid,
                         sy.tp, 1 + g, lat);
          done = true;
        }
      }
      if constexpr (kLattice == kStreamKernel || kLattice == kMixedKernel) {
        if (!done && sy.mode == kModeStreamed) {
          Real* lat = reinterpret_cast<Real*>(
              static_cast<unsigned char*>(P.lattice) +
              (static_cast<int64_t>(blockIdx.x) * P.lattice_groups + g) * P.lattice_stride);
          if constexpr (kLattice == kMixedKernel) {
            // batches of uneven sizes: the streamed size of the benchmark's
            // batch (L = 32) with compile-time rows
            if (sy.L == 32 && sy.tp == 8 * 32)
              run_path_streamed<Real, 32, 16>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes,
                                              tid, sy.tp, 1 + g, lat);
            else if (sy.L == 32 && sy.tp == 4 * 32)
              run_path_streamed<Real, 32, 8>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes,
                                             tid, sy.tp, 1 + g, lat);
            else
              run_path_streamed<Real, 0, 0>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes,
                                            tid, sy.tp, 1 + g, lat);
          } else {
            run_path_streamed<Real, 0, 0>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes, tid,
                                          sy.tp, 1 + g, lat);
          }
          done = true;
        }
      }
      if (!done)
        dispatch_path<Real, kLattice>(sy, it.sys, it.path0 + g, P, smem + g * sy.slice_bytes, tid,
                                      sy.tp, 1 + g);
    }
  }
}

}  // namespace mpk
