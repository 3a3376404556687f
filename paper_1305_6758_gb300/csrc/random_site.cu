// The paper's literal sweep order (Sec. 2.2): a lattice sweep is N Metropolis
// attempts at randomly chosen sites, so consecutive attempts of one path may
// touch neighbouring sites and a path is strictly sequential.  The parallelism
// is across paths only: one thread per path, its lattice in HBM (it cannot
// share an SM's shared memory with enough other paths to fill it).
//
// Attempt a of sweep s of a path draws one counter (a, s, path, 2 | sys<<8):
// the site is the cell of width 1/N holding u(r3), i = floor((2 r3 + 1) N / 2^33)
// in integer arithmetic, and r0, r1, r2 drive the trial move and the accept
// test exactly as in the checkerboard kernels.  After every measurement sweep
// the energy is a bond loop (+x, +y, +z bonds of each site, in site order) and
// m the spin sum, both in the working precision, as in the oracle's
// definition; the FP64 form evaluates them term by term without fused
// multiply-adds so that its records follow the oracle's arithmetic.
//
// Lattice layout: element (site i, path p) of system k at
// spin_offset[k] / 3 + i * P_k + p, so the threads of a warp (consecutive
// paths) read consecutive elements when they visit the same site (start,
// measurement).  FP32: one float4 (x, y, z, unused) per element; FP64: three
// planes of doubles.
#include "kernels.h"
#include "sweep.cuh"

namespace mpk {

namespace {

constexpr uint32_t kTagSite = 2u;

template <typename Real>
struct SiteStore;

template <>
struct SiteStore<float> {
  float4* a;
  __device__ void ld(int64_t e, float& x, float& y, float& z) const {
    const float4 v = a[e];
    x = v.x;
    y = v.y;
    z = v.z;
  }
  __device__ void st(int64_t e, float x, float y, float z) const { a[e] = make_float4(x, y, z, 0.f); }
  __device__ float dot(float ax, float ay, float az, float bx, float by, float bz) const {
    return ax * bx + ay * by + az * bz;
  }
  __device__ float add(float a_, float b) const { return a_ + b; }
};

template <>
struct SiteStore<double> {
  double* a;
  int64_t plane;  // elements per component plane
  __device__ void ld(int64_t e, double& x, double& y, double& z) const {
    x = a[e];
    y = a[plane + e];
    z = a[2 * plane + e];
  }
  __device__ void st(int64_t e, double x, double y, double z) const {
    a[e] = x;
    a[plane + e] = y;
    a[2 * plane + e] = z;
  }
  __device__ double dot(double ax, double ay, double az, double bx, double by, double bz) const {
    return __dadd_rn(__dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)), __dmul_rn(az, bz));
  }
  __device__ double add(double a_, double b) const { return __dadd_rn(a_, b); }
};

// Neighbours of site i in the fixed order +x, -x, +y, -y, +z, -z (simple
// cubic, periodic) or i-1, i+1 where they exist (open chain).
__device__ __forceinline__ int neighbours(int lattice, int L, int i, int* nb) {
  if (lattice == MP_LATTICE_CHAIN) {
    int k = 0;
    if (i > 0) nb[k++] = i - 1;
    if (i < L - 1) nb[k++] = i + 1;
    return k;
  }
  const int x = i % L, t = i / L, y = t % L, z = t / L;
  const int LL = L * L;
  nb[0] = i + (x == L - 1 ? 1 - L : 1);
  nb[1] = i + (x == 0 ? L - 1 : -1);
  nb[2] = i + (y == L - 1 ? L - LL : L);
  nb[3] = i + (y == 0 ? LL - L : -L);
  nb[4] = i + (z == L - 1 ? -(L - 1) * LL : LL);
  nb[5] = i + (z == 0 ? (L - 1) * LL : -LL);
  return 6;
}

template <typename Real>
__global__ void __launch_bounds__(128) random_site_kernel(const SweepParams P, int n_systems,
                                                          int64_t total_paths, void* lattice,
                                                          int64_t plane) {
  using A = Arith<Real>;
  const int64_t gp = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gp >= total_paths) return;
  // the system of global path gp: the last one whose first path is <= gp
  int lo = 0, hi = n_systems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.systems[mid].rec_offset <= gp) lo = mid;
    else hi = mid - 1;
  }
  const int k = lo;
  const DevSystem sy = P.systems[k];
  const int64_t path = gp - sy.rec_offset;
  const int64_t Pk = sy.n_paths;
  const int N = sy.N, L = sy.L;
  const int64_t base = P.spin_offset[k] / 3 + path;  // element of site 0
  SiteStore<Real> S;
  if constexpr (sizeof(Real) == 4) {
    S.a = static_cast<float4*>(lattice);
  } else {
    S.a = static_cast<double*>(lattice);
    S.plane = plane;
  }
  auto el = [&](int i) { return base + static_cast<int64_t>(i) * Pk; };
  const uint32_t c2 = static_cast<uint32_t>(sy.path_begin + path);  // path id
  const uint32_t sys_hi = static_cast<uint32_t>(k) << 8;
  const int init = path_init_mode(P.init_mode, path, Pk);
  for (int i = 0; i < N; ++i) {
    Real x, y, z;
    initial_spin<Real>(static_cast<uint32_t>(i), c2, kTagInit | sys_hi, P, init, x, y, z);
    S.st(el(i), x, y, z);
  }
  const Real J = static_cast<Real>(sy.J), hf = static_cast<Real>(sy.h);
  const Real bp = A::beta_param(sy.beta);
  double acc[kAccDoubles];
#pragma unroll
  for (int q = 0; q < kAccDoubles; ++q) acc[q] = 0.0;
  int64_t accepted = 0;
  const int64_t S_total = P.n_therm + P.n_meas;
  for (int64_t s = 0; s < S_total; ++s) {
    const PhiloxPrefix pre = philox_prefix(static_cast<uint32_t>(s), c2, kTagSite | sys_hi, P.key);
    for (int a = 0; a < N; ++a) {
      const Philox4 r = philox4x32_10(static_cast<uint32_t>(a), pre, P.key);
      const int i = static_cast<int>(((static_cast<uint64_t>(r.w) * 2u + 1u) *
                                      static_cast<uint64_t>(N)) >> 33);
      int nb[6];
      const int nn = neighbours(sy.lattice, L, i, nb);
      Real hx = Real(0), hy = Real(0), hz = Real(0);
      for (int j = 0; j < nn; ++j) {
        Real x, y, z;
        S.ld(el(nb[j]), x, y, z);
        hx = S.add(hx, x);
        hy = S.add(hy, y);
        hz = S.add(hz, z);
      }
      Real tx, ty, tz, ax, ay, az;
      A::trial(r.x, r.y, tx, ty, tz);
      S.ld(el(i), ax, ay, az);
      if (A::accept_move(tx - ax, ty - ay, tz - az, hx, hy, hz, J, hf, bp, r.z)) {
        S.st(el(i), tx, ty, tz);
        ++accepted;
      }
    }
    if (s < P.n_therm) continue;
    // measurement: bond loop and spin sum, in site order
    Real bonds = Real(0), sx = Real(0), sy_ = Real(0), sz = Real(0);
    for (int i = 0; i < N; ++i) {
      Real ax, ay, az;
      S.ld(el(i), ax, ay, az);
      sx = S.add(sx, ax);
      sy_ = S.add(sy_, ay);
      sz = S.add(sz, az);
      if (sy.lattice == MP_LATTICE_CHAIN) {
        if (i + 1 < N) {
          Real bx, by, bz;
          S.ld(el(i + 1), bx, by, bz);
          bonds = S.add(bonds, S.dot(ax, ay, az, bx, by, bz));
        }
        continue;
      }
      int nb[6];
      neighbours(MP_LATTICE_SC, L, i, nb);
#pragma unroll
      for (int d = 0; d < 3; ++d) {  // +x, +y, +z
        Real bx, by, bz;
        S.ld(el(nb[2 * d]), bx, by, bz);
        bonds = S.add(bonds, S.dot(ax, ay, az, bx, by, bz));
      }
    }
    const double dN = static_cast<double>(N);
    double e, mx, my, mz;
    if constexpr (sizeof(Real) == 8) {
      e = __ddiv_rn(__dsub_rn(__dmul_rn(-sy.J, bonds), __dmul_rn(sy.h, sz)), dN);
      mx = __ddiv_rn(sx, dN);
      my = __ddiv_rn(sy_, dN);
      mz = __ddiv_rn(sz, dN);
    } else {
      e = static_cast<double>(-J * bonds - hf * sz) / dN;
      mx = static_cast<double>(sx) / dN;
      my = static_cast<double>(sy_) / dN;
      mz = static_cast<double>(sz) / dN;
    }
    const double m = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(mx, mx), __dmul_rn(my, my)), __dmul_rn(mz, mz)));
    acc[MP_R_E] = __dadd_rn(acc[MP_R_E], e);
    acc[MP_R_E2] = __dadd_rn(acc[MP_R_E2], __dmul_rn(e, e));
    acc[MP_R_M] = __dadd_rn(acc[MP_R_M], m);
    acc[MP_R_M2] = __dadd_rn(acc[MP_R_M2], __dmul_rn(m, m));
    acc[MP_R_M4] = __dadd_rn(acc[MP_R_M4], __dmul_rn(__dmul_rn(__dmul_rn(m, m), m), m));
    acc[MP_R_MX] = __dadd_rn(acc[MP_R_MX], mx);
    acc[MP_R_MY] = __dadd_rn(acc[MP_R_MY], my);
    acc[MP_R_MZ] = __dadd_rn(acc[MP_R_MZ], mz);
    acc[MP_R_MZ2] = __dadd_rn(acc[MP_R_MZ2], __dmul_rn(mz, mz));
    acc[MP_R_AMZ] = __dadd_rn(acc[MP_R_AMZ], fabs(mz));
    acc[MP_R_EM] = __dadd_rn(acc[MP_R_EM], __dmul_rn(e, m));
    acc[MP_R_EMZ] = __dadd_rn(acc[MP_R_EMZ], __dmul_rn(e, mz));
    acc[MP_R_MMZ] = __dadd_rn(acc[MP_R_MMZ], __dmul_rn(m, mz));
    if (s == S_total - 1) {
      acc[MP_R_FMX] = mx;
      acc[MP_R_FMY] = my;
      acc[MP_R_FMZ] = mz;
      acc[MP_R_FE] = e;
    }
  }
  double* rec = P.records + gp * MP_NREC;
  const double n_meas = static_cast<double>(P.n_meas);
#pragma unroll
  for (int q = MP_R_E; q <= MP_R_MMZ; ++q) rec[q] = __ddiv_rn(acc[q], n_meas);
#pragma unroll
  for (int q = MP_R_FMX; q <= MP_R_FE; ++q) rec[q] = acc[q];
  rec[MP_R_ACC] = static_cast<double>(accepted) / (static_cast<double>(S_total) * static_cast<double>(N));
  double worst = 0.0;
  double* out = P.spins ? P.spins + P.spin_offset[k] + path * 3 * static_cast<int64_t>(N) : nullptr;
  for (int i = 0; i < N; ++i) {
    Real x, y, z;
    S.ld(el(i), x, y, z);
    worst = fmax(worst, static_cast<double>(fabs(sqrt(x * x + y * y + z * z) - Real(1))));
    if (out) {
      out[3 * i + 0] = x;
      out[3 * i + 1] = y;
      out[3 * i + 2] = z;
    }
  }
  rec[MP_R_NORM] = worst;
  rec[MP_R_SPARE] = 0.0;
}

}  // namespace

// Lattice bytes per site and path of the random-site kernels.
int random_site_bytes_per_site(int precision) { return precision == MP_FP64 ? 24 : 16; }

// elements = sites x paths over all systems (FP64: the size of one component plane)
cudaError_t launch_random_site(int precision, const SweepParams& p, int n_systems, int64_t total_paths,
                               void* lattice, int64_t elements, cudaStream_t st) {
  const int threads = 128;
  const int64_t blocks = (total_paths + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (precision == MP_FP64)
    random_site_kernel<double><<<static_cast<unsigned>(blocks), threads, 0, st>>>(
        p, n_systems, total_paths, lattice, elements);
  else
    random_site_kernel<float><<<static_cast<unsigned>(blocks), threads, 0, st>>>(
        p, n_systems, total_paths, lattice, elements);
  return cudaGetLastError();
}

}  // namespace mpk
