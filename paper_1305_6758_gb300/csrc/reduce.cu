// Cross-path reduction: per-path records -> ensemble estimates (one CTA per
// system, FP64 throughout), the covariance backward, and a Philox kernel for
// stream checks.
//
// Estimates follow Sec. 2.2 of Rakic et al.: the MC average over paths,
// Eq. (MCAV); chi and C_V from the fluctuation formulas, Eq. (cv); the Binder
// cumulant, Eq. (kum); the coefficient of variation of a mean, Eq. (eq:cv);
// and the distribution coefficient of the normal Q-Q line fit, Eq.
// (dist-coefficient) of Sec. 3.  Standard errors of derived quantities are
// delete-one jackknife over paths (paths are independent, so no blocking).
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "philox.cuh"

namespace mpk {

static_assert(sizeof(mp_estimates_t) == MP_NEST * sizeof(double), "estimates layout");

constexpr int kRedThreads = 512;
constexpr int kNumMean = 13;  // record fields MP_R_E .. MP_R_MMZ
constexpr int kNumDerived = 9;

// Sum V values over the CTA; every thread receives the totals.
template <int V>
__device__ void block_sum(double (&v)[V], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < V; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < V; ++k) scratch[warp * V + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < V; ++k) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += scratch[w * V + k];
    v[k] = t;
  }
  __syncthreads();
}

__device__ double block_max(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = scratch[0];
  for (int w = 1; w < nw; ++w) t = fmax(t, scratch[w]);
  __syncthreads();
  return t;
}

// chi, C_V, U_L and the six fluctuation derivatives from pooled means
// (indexed by MP_R_*).  Under the weight exp(-beta N e):
//   d<A>/dbeta = -N cov(A, e),   d<A>/dh = <dA/dh> + beta N cov(A, m_z),
// and of A in {e, |m|, m_z} only e = (-J E_bonds - h M_z)/N depends on h
// itself (de/dh = -m_z).
__device__ void derived(const double* mu, double N, double beta, double* th) {
  const double e = mu[MP_R_E], e2 = mu[MP_R_E2], m = mu[MP_R_M], m2 = mu[MP_R_M2];
  const double m4 = mu[MP_R_M4], mz = mu[MP_R_MZ], mz2 = mu[MP_R_MZ2];
  const double em = mu[MP_R_EM], emz = mu[MP_R_EMZ], mmz = mu[MP_R_MMZ];
  th[0] = N * beta * (m2 - m * m);          // chi
  th[1] = N * beta * beta * (e2 - e * e);   // C_V
  th[2] = 1.0 - m4 / (3.0 * m2 * m2);       // Binder U_L
  th[3] = -N * (e2 - e * e);                // d<e>/dbeta
  th[4] = -N * (em - m * e);                // d<|m|>/dbeta
  th[5] = -N * (emz - mz * e);              // d<m_z>/dbeta
  th[6] = beta * N * (emz - e * mz) - mz;   // d<e>/dh: e's own field term adds -<m_z>
  th[7] = beta * N * (mmz - m * mz);        // d<|m|>/dh
  th[8] = beta * N * (mz2 - mz * mz);       // d<m_z>/dh
}

// Eq. (dist-coefficient) of one record field: sort the P values (bitonic, in
// `keys`: shared memory up to MP_R_MAX_PATHS paths, a device buffer of at
// least the next power of two above P beyond), fit them to the normal
// quantiles at (i - 1/2)/P by least squares;
// r = 1 - SS_res / ((P-1) sigma^2) = S_xq^2 / (S_xx S_qq).
__device__ double distribution_coefficient(const double* rec, int64_t P, int field, double mean,
                                           double* keys, double* scratch) {
  int n = 1;
  while (n < P) n <<= 1;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    keys[i] = i < P ? rec[static_cast<int64_t>(i) * MP_NREC + field] : INFINITY;
  __syncthreads();
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const double a = keys[i], b = keys[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            keys[i] = b;
            keys[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  const double invP = 1.0 / static_cast<double>(P);
  double qs[1] = {0.0};
  for (int i = threadIdx.x; i < P; i += blockDim.x) qs[0] += normcdfinv((i + 0.5) * invP);
  block_sum<1>(qs, scratch);
  const double qbar = qs[0] * invP;
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double dx = keys[i] - mean;
    const double dq = normcdfinv((i + 0.5) * invP) - qbar;
    s[0] += dx * dx;
    s[1] += dq * dq;
    s[2] += dx * dq;
  }
  block_sum<3>(s, scratch);
  if (!(s[0] > 0.0) || !(s[1] > 0.0)) return NAN;
  return s[2] * s[2] / (s[0] * s[1]);
}

__global__ void __launch_bounds__(kRedThreads) reduce_kernel(const ReduceParams p) {
  extern __shared__ __align__(16) double keys[];
  __shared__ double scratch[32 * 16];
  const int sidx = blockIdx.x;
  const DevSystem sy = p.systems[sidx];
  const int64_t P = sy.n_paths;
  const double* rec = p.records + sy.rec_offset * MP_NREC;
  const double N = static_cast<double>(sy.N), beta = sy.beta;
  const double invP = 1.0 / static_cast<double>(P);

  // pass 1: means of the record fields, and the acceptance mean
  double sum[kNumMean + 1];
#pragma unroll
  for (int k = 0; k <= kNumMean; ++k) sum[k] = 0.0;
  double worst = 0.0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double* r = rec + i * MP_NREC;
#pragma unroll
    for (int k = 0; k < kNumMean; ++k) sum[k] += r[k];
    sum[kNumMean] += r[MP_R_ACC];
    worst = fmax(worst, r[MP_R_NORM]);
  }
  block_sum<kNumMean + 1>(sum, scratch);
  worst = block_max(worst, scratch);
  double mu[kNumMean + 1];
#pragma unroll
  for (int k = 0; k <= kNumMean; ++k) mu[k] = sum[k] * invP;

  // pass 2: sample variances for the standard errors of the means
  double var[kNumMean + 1];
#pragma unroll
  for (int k = 0; k <= kNumMean; ++k) var[k] = 0.0;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double* r = rec + i * MP_NREC;
#pragma unroll
    for (int k = 0; k < kNumMean; ++k) {
      const double d = r[k] - mu[k];
      var[k] += d * d;
    }
    const double d = r[MP_R_ACC] - mu[kNumMean];
    var[kNumMean] += d * d;
  }
  block_sum<kNumMean + 1>(var, scratch);

  // passes 3 and 4: delete-one jackknife of the derived quantities
  double th_full[kNumDerived];
  derived(mu, N, beta, th_full);
  double jk_mean[kNumDerived], jk_var[kNumDerived];
#pragma unroll
  for (int k = 0; k < kNumDerived; ++k) {
    jk_mean[k] = 0.0;
    jk_var[k] = 0.0;
  }
  const bool jk = P >= 2;
  if (jk) {
    const double invPm1 = 1.0 / static_cast<double>(P - 1);
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
      const double* r = rec + i * MP_NREC;
      double loo[kNumMean], th[kNumDerived];
#pragma unroll
      for (int k = 0; k < kNumMean; ++k) loo[k] = (sum[k] - r[k]) * invPm1;
      derived(loo, N, beta, th);
#pragma unroll
      for (int k = 0; k < kNumDerived; ++k) jk_mean[k] += th[k];
    }
    block_sum<kNumDerived>(jk_mean, scratch);
#pragma unroll
    for (int k = 0; k < kNumDerived; ++k) jk_mean[k] *= invP;
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
      const double* r = rec + i * MP_NREC;
      double loo[kNumMean], th[kNumDerived];
#pragma unroll
      for (int k = 0; k < kNumMean; ++k) loo[k] = (sum[k] - r[k]) * invPm1;
      derived(loo, N, beta, th);
#pragma unroll
      for (int k = 0; k < kNumDerived; ++k) {
        const double d = th[k] - jk_mean[k];
        jk_var[k] += d * d;
      }
    }
    block_sum<kNumDerived>(jk_var, scratch);
  }

  // The two halves of the paths (Sec. 4's two-start check): paths
  // 0 .. Pa-1 and Pa .. P-1 with Pa = ceil(P/2); sums, then variances, of e
  // and |m| over each half.
  const int64_t Pa = P - P / 2, Pb = P / 2;
  double hs[4] = {0.0, 0.0, 0.0, 0.0};  // e_a, m_a, e_b, m_b
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double* r = rec + i * MP_NREC;
    const bool a = i < Pa;
    hs[0] += a ? r[MP_R_E] : 0.0;
    hs[1] += a ? r[MP_R_M] : 0.0;
    hs[2] += a ? 0.0 : r[MP_R_E];
    hs[3] += a ? 0.0 : r[MP_R_M];
  }
  block_sum<4>(hs, scratch);
  const double hmu[4] = {hs[0] / Pa, hs[1] / Pa, Pb ? hs[2] / Pb : NAN, Pb ? hs[3] / Pb : NAN};
  double hv[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double* r = rec + i * MP_NREC;
    const bool a = i < Pa;
    const double de = r[MP_R_E] - (a ? hmu[0] : hmu[2]), dm = r[MP_R_M] - (a ? hmu[1] : hmu[3]);
    hv[0] += a ? de * de : 0.0;
    hv[1] += a ? dm * dm : 0.0;
    hv[2] += a ? 0.0 : de * de;
    hv[3] += a ? 0.0 : dm * dm;
  }
  block_sum<4>(hv, scratch);

  // pass 5: distribution coefficients of the per-path outputs
  const int rfield[6] = {MP_R_E, MP_R_M, MP_R_MX, MP_R_MY, MP_R_MZ, MP_R_AMZ};
  double* sort_keys = P <= MP_R_MAX_PATHS ? keys
                      : (p.sort_buf != nullptr && P <= (int64_t{1} << 30)) ? p.sort_buf + 2 * sy.rec_offset
                                                                           : nullptr;
  double rcoef[6];
  for (int f = 0; f < 6; ++f) {
    rcoef[f] = (P >= 3 && sort_keys != nullptr)
                   ? distribution_coefficient(rec, P, rfield[f], mu[rfield[f]], sort_keys, scratch)
                   : NAN;
  }

  if (threadIdx.x == 0) {
    mp_estimates_t* o = reinterpret_cast<mp_estimates_t*>(p.est + sidx * MP_NEST);
    const double sq = P >= 2 ? 1.0 / sqrt(static_cast<double>(P) * static_cast<double>(P - 1)) : NAN;
    auto se = [&](int k) { return sqrt(var[k]) * sq; };
    const double jks = P >= 2 ? static_cast<double>(P - 1) * invP : NAN;
    auto jse = [&](int k) { return jk ? sqrt(jks * jk_var[k]) : NAN; };
    o->n_paths = static_cast<double>(P);
    o->N = N;
    o->T = sy.T;
    o->n_meas = static_cast<double>(p.n_meas);
    o->e = mu[MP_R_E];       o->e_se = se(MP_R_E);
    o->e2 = mu[MP_R_E2];     o->e2_se = se(MP_R_E2);
    o->m = mu[MP_R_M];       o->m_se = se(MP_R_M);
    o->m2 = mu[MP_R_M2];     o->m2_se = se(MP_R_M2);
    o->m4 = mu[MP_R_M4];     o->m4_se = se(MP_R_M4);
    o->mx = mu[MP_R_MX];     o->mx_se = se(MP_R_MX);
    o->my = mu[MP_R_MY];     o->my_se = se(MP_R_MY);
    o->mz = mu[MP_R_MZ];     o->mz_se = se(MP_R_MZ);
    o->mz2 = mu[MP_R_MZ2];   o->mz2_se = se(MP_R_MZ2);
    o->amz = mu[MP_R_AMZ];   o->amz_se = se(MP_R_AMZ);
    o->acc = mu[kNumMean];   o->acc_se = se(kNumMean);
    o->chi = th_full[0];       o->chi_se = jse(0);
    o->cv = th_full[1];        o->cv_se = jse(1);
    o->binder = th_full[2];    o->binder_se = jse(2);
    o->de_dbeta = th_full[3];  o->de_dbeta_se = jse(3);
    o->dm_dbeta = th_full[4];  o->dm_dbeta_se = jse(4);
    o->dmz_dbeta = th_full[5]; o->dmz_dbeta_se = jse(5);
    o->de_dh = th_full[6];     o->de_dh_se = jse(6);
    o->dm_dh = th_full[7];     o->dm_dh_se = jse(7);
    o->dmz_dh = th_full[8];    o->dmz_dh_se = jse(8);
    o->cv_m = o->m_se / o->m;
    o->r_e = rcoef[0];
    o->r_m = rcoef[1];
    o->r_mx = rcoef[2];
    o->r_my = rcoef[3];
    o->r_mz = rcoef[4];
    o->r_amz = rcoef[5];
    o->attempts = N * static_cast<double>(P) * static_cast<double>(p.n_therm + p.n_meas);
    o->norm_max = worst;
    auto hse = [&](int k, int64_t n) {
      return n >= 2 ? sqrt(hv[k] / (static_cast<double>(n) * static_cast<double>(n - 1))) : NAN;
    };
    o->e_a = hmu[0];  o->e_a_se = hse(0, Pa);
    o->m_a = hmu[1];  o->m_a_se = hse(1, Pa);
    o->e_b = hmu[2];  o->e_b_se = hse(2, Pb);
    o->m_b = hmu[3];  o->m_b_se = hse(3, Pb);
    const double ze = fabs(o->e_a - o->e_b) / sqrt(o->e_a_se * o->e_a_se + o->e_b_se * o->e_b_se);
    const double zm = fabs(o->m_a - o->m_b) / sqrt(o->m_a_se * o->m_a_se + o->m_b_se * o->m_b_se);
    o->start_z = fmax(ze, zm);  // an undefined ratio (0/0) is skipped
    o->elapsed_s = NAN;  // the host fills it in from the run's events
    o->reserved[0] = 0.0;
  }
}

// Covariance backward: for each system, with upstream gradients (g_e, g_m) of
// (<e>, <|m|>),  dL/dbeta = -N [g_e cov(e, e) + g_m cov(|m|, e)]  and
// dL/dh = beta N [g_e cov(e, m_z) + g_m cov(|m|, m_z)] - g_e <m_z> (the last
// term from the field part of e), covariances of the pooled per-path moments
// (the C_V / chi estimators of Eq. (cv)).
__global__ void __launch_bounds__(kRedThreads) backward_kernel(const BackwardParams p) {
  __shared__ double scratch[32 * 8];
  const int sidx = blockIdx.x;
  const DevSystem sy = p.systems[sidx];
  const int64_t P = sy.n_paths;
  const double* rec = p.records + sy.rec_offset * MP_NREC;
  double s[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const double* r = rec + i * MP_NREC;
    s[0] += r[MP_R_E];
    s[1] += r[MP_R_E2];
    s[2] += r[MP_R_M];
    s[3] += r[MP_R_EM];
    s[4] += r[MP_R_MZ];
    s[5] += r[MP_R_EMZ];
    s[6] += r[MP_R_MMZ];
  }
  block_sum<7>(s, scratch);
  if (threadIdx.x == 0) {
    const double inv = 1.0 / static_cast<double>(P);
    const double e = s[0] * inv, e2 = s[1] * inv, m = s[2] * inv, em = s[3] * inv;
    const double mz = s[4] * inv, emz = s[5] * inv, mmz = s[6] * inv;
    const double N = static_cast<double>(sy.N), beta = sy.beta;
    const double ge = p.g_e[sidx], gm = p.g_m[sidx];
    p.grad_beta[sidx] = -N * (ge * (e2 - e * e) + gm * (em - m * e));
    p.grad_h[sidx] = beta * N * (ge * (emz - e * mz) + gm * (mmz - m * mz)) - ge * mz;
  }
}

__global__ void philox_kernel(const uint32_t* ctr, int64_t n, const PhiloxKeys key, uint32_t* out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const Philox4 r = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], key);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
  }
}

cudaError_t launch_reduce(const ReduceParams& p, int n_systems, int64_t max_paths, cudaStream_t st) {
  int n = 1;
  while (n < max_paths && n < MP_R_MAX_PATHS) n <<= 1;
  const int smem = static_cast<int>(n * sizeof(double));
  reduce_kernel<<<n_systems, kRedThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t reduce_prepare() {
  return cudaFuncSetAttribute(reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              MP_R_MAX_PATHS * static_cast<int>(sizeof(double)));
}

cudaError_t launch_backward(const BackwardParams& p, int n_systems, cudaStream_t st) {
  backward_kernel<<<n_systems, kRedThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = (n + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  philox_kernel<<<static_cast<int>(blocks), threads, 0, st>>>(ctr, n, philox_round_keys(seed), out);
  return cudaGetLastError();
}

}  // namespace mpk
