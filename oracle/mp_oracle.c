/*
 * Multipath Metropolis oracle for the classical O(3) Heisenberg model.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 CPU statement
 * of what the multipath method computes.  It shares no code with the CUDA
 * library; only tests, the smoke check and the CPU-baseline leg of the bench
 * may load it.  Nothing on the product path calls it.
 *
 * What it follows (Rakic et al., "Multipath Metropolis Simulation of
 * Classical Heisenberg Model"):
 *   - Eq. (1): H = -(J/2) sum_n sum_lambda S_n . S_{n+lambda} on a periodic
 *     simple-cubic lattice with N = L^3 sites (Sec. 2.1).  A Zeeman term
 *     -h sum_n S^z_n is added (the paper has none; h = 0 reproduces it).
 *   - Eq. (2): unit spins S = (sin t cos f, sin t sin f, cos t) (Sec. 2.1).
 *   - Sec. 2.2: Metropolis single spin-flip updates, a lattice sweep of N
 *     attempts, many independent simulation paths from random initial states,
 *     and per-path outputs {M^x, M^y, M^z, H} per lattice site.
 *   - Appendix A: the same scheme on the square-lattice Ising model
 *     (run_path_ising, with its own readings).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - trial move: a fresh direction uniform on the sphere, independent of the
 *     old spin (cos t uniform in (-1,1), f uniform in (0, 2 pi));
 *   - acceptance: accept when dE <= 0, else accept iff u < exp(-beta dE);
 *   - site order: checkerboard (colour (x+y+z) mod 2 = 0 first, then 1, each
 *     colour in increasing site index).  The paper's "N randomly chosen sites"
 *     order is order_mode = 1 (one counter per attempt gives the site and the
 *     move; see run_path);
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *     key = (seed lo, seed hi) and counter = (site, sweep, path, tag | sys<<8);
 *   - per-path output: the mean over n_meas measurement sweeps (n_meas = 1 is
 *     the paper's single final-state output); the final state is kept too.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread -o libmp_oracle.so
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_SC 0    /* periodic simple cubic, N = L^3 */
#define OR_CHAIN 1 /* open chain, N = L */
#define OR_ISING 2 /* Appendix A: periodic square lattice of Ising spins, N = L^2 */

#define OR_INIT_SPHERE 0  /* uniform on the sphere (Sec. 4 "uniform state") */
#define OR_INIT_ANGLES 1  /* theta, phi each uniform ("both angles random") */
#define OR_INIT_ORDERED 2 /* all spins along +z (Sec. 5 ordered start) */
#define OR_TWO_START 0x100 /* or-ed into init_mode: second half of paths ordered */

#define OR_ORDER_CHECKER 0
#define OR_ORDER_RANDOM 1

#define OR_TAG_UPDATE 0u
#define OR_TAG_INIT 1u
#define OR_TAG_SITE 2u
#define OR_TAG_ISING 4u /* Ising updates: tag 4 + colour */

/* per-path record layout: means over the measurement sweeps, then the final
 * state (the paper's SP output), then bookkeeping */
enum {
  R_E = 0, R_E2, R_M, R_M2, R_M4, R_MX, R_MY, R_MZ, R_MZ2, R_AMZ,
  R_EM, R_EMZ, R_MMZ, R_FMX, R_FMY, R_FMZ, R_FE, R_ACC, R_NORM, R_SPARE,
  NREC
};

typedef struct {
  int32_t lattice;
  int32_t L;
  double T, J, h;
  int64_t n_paths;
  int64_t path_begin;
  int64_t path_count;
} oracle_system;

/* ---------------------------------------------------------------- Philox --
 * Philox4x32-10, SC'11: each round multiplies words 0 and 2 by the two round
 * multipliers, takes high and low halves, and mixes in the other two words
 * and the round key; the key is bumped by the two Weyl constants between
 * rounds.  Ten rounds. */
static const uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
static const uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

void oracle_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                   uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PH_M0 * x0;
    uint64_t p1 = (uint64_t)PH_M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PH_W0;
    k1 += PH_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in the open interval (0,1), exact in double */
static double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------- geometry --
 * Site i = x + L*(y + L*z).  Neighbour order is fixed: +x, -x, +y, -y, +z, -z
 * with periodic wrap; the chain has i-1 then i+1 where they exist. */
static int64_t n_sites(int lattice, int L) {
  if (lattice == OR_ISING) return (int64_t)L * L;
  return lattice == OR_SC ? (int64_t)L * L * L : (int64_t)L;
}

static int neighbours(int lattice, int L, int64_t i, int64_t nb[6]) {
  if (lattice == OR_CHAIN) {
    int k = 0;
    if (i > 0) nb[k++] = i - 1;
    if (i < L - 1) nb[k++] = i + 1;
    return k;
  }
  int64_t x = i % L, y = (i / L) % L, z = i / ((int64_t)L * L);
  int64_t xp = (x + 1) % L, xm = (x + L - 1) % L;
  int64_t yp = (y + 1) % L, ym = (y + L - 1) % L;
  int64_t zp = (z + 1) % L, zm = (z + L - 1) % L;
  nb[0] = xp + L * (y + L * z);
  nb[1] = xm + L * (y + L * z);
  nb[2] = x + L * (yp + L * z);
  nb[3] = x + L * (ym + L * z);
  nb[4] = x + L * (y + L * zp);
  nb[5] = x + L * (y + L * zm);
  return 6;
}

static int colour(int lattice, int L, int64_t i) {
  if (lattice == OR_CHAIN) return (int)(i & 1);
  int64_t x = i % L, y = (i / L) % L, z = i / ((int64_t)L * L);
  return (int)((x + y + z) & 1);
}

/* Unit vector from two uniforms: cos(theta) = 2 u0 - 1, phi = 2 pi u1
 * (Eq. 2 with cos(theta) uniform, i.e. uniform on the sphere). */
static void sphere_point(double u0, double u1, double s[3]) {
  double z = 2.0 * u0 - 1.0;
  double r = sqrt((1.0 - z) * (1.0 + z));
  double phi = 2.0 * M_PI * u1;
  s[0] = r * cos(phi);
  s[1] = r * sin(phi);
  s[2] = z;
}

/* Total energy by a direct bond loop, Eq. (1) plus the Zeeman term.  On the
 * simple-cubic lattice each site owns its +x, +y, +z bonds, so every bond of
 * the double sum in Eq. (1) is visited once after the factor 1/2. */
double oracle_energy(int lattice, int L, double J, double h, const double* s) {
  int64_t N = n_sites(lattice, L);
  double bonds = 0.0, sz = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const double* a = s + 3 * i;
    sz += a[2];
    if (lattice == OR_CHAIN) {
      if (i + 1 < N) {
        const double* b = s + 3 * (i + 1);
        bonds += a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
      }
      continue;
    }
    int64_t x = i % L, y = (i / L) % L, z = i / ((int64_t)L * L);
    int64_t up[3] = {(x + 1) % L + L * (y + L * z), x + L * ((y + 1) % L + L * z),
                     x + L * (y + L * ((z + 1) % L))};
    for (int d = 0; d < 3; ++d) {
      const double* b = s + 3 * up[d];
      bonds += a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    }
  }
  return -J * bonds - h * sz;
}

/* Energy change of replacing spin i by t, from the local field of its
 * neighbours: dE = -J (t - S_i) . h_loc - h (t_z - S_i,z). */
double oracle_delta_e(int lattice, int L, double J, double h, const double* s,
                      int64_t i, const double* t) {
  int64_t nb[6];
  int k = neighbours(lattice, L, i, nb);
  double hx = 0.0, hy = 0.0, hz = 0.0;
  for (int j = 0; j < k; ++j) {
    hx += s[3 * nb[j] + 0];
    hy += s[3 * nb[j] + 1];
    hz += s[3 * nb[j] + 2];
  }
  const double* a = s + 3 * i;
  double dot = (t[0] - a[0]) * hx + (t[1] - a[1]) * hy + (t[2] - a[2]) * hz;
  return -J * dot - h * (t[2] - a[2]);
}

/* One Metropolis attempt at site i with the words r of its update counter:
 * trial from r[0], r[1]; accept when dE <= 0, else iff u(r[2]) < exp(-beta dE).
 * Returns 1 when the trial was accepted. */
static int metropolis(int lat, int L, double J, double hf, double beta, double* s,
                      int64_t i, const uint32_t r[4]) {
  double t[3];
  sphere_point(u01(r[0]), u01(r[1]), t);
  double dE = oracle_delta_e(lat, L, J, hf, s, i, t);
  if (dE <= 0.0 || u01(r[2]) < exp(-beta * dE)) {
    s[3 * i + 0] = t[0]; s[3 * i + 1] = t[1]; s[3 * i + 2] = t[2];
    return 1;
  }
  return 0;
}

/* Sec. 2.2: the random initial state of a path (or the ordered start of
 * Sec. 5), from the init stream (tag 1, sweep 0) of each site. */
static void init_state(int64_t N, uint32_t path, uint32_t sys_hi, uint32_t k0, uint32_t k1,
                       int init_mode, double* s) {
  uint32_t r[4];
  for (int64_t i = 0; i < N; ++i) {
    oracle_philox((uint32_t)i, 0u, path, OR_TAG_INIT | sys_hi, k0, k1, r);
    if (init_mode == OR_INIT_ORDERED) {
      s[3 * i + 0] = 0.0; s[3 * i + 1] = 0.0; s[3 * i + 2] = 1.0;
    } else if (init_mode == OR_INIT_ANGLES) {
      double th = M_PI * u01(r[0]), ph = 2.0 * M_PI * u01(r[1]);
      s[3 * i + 0] = sin(th) * cos(ph);
      s[3 * i + 1] = sin(th) * sin(ph);
      s[3 * i + 2] = cos(th);
    } else {
      sphere_point(u01(r[0]), u01(r[1]), s + 3 * i);
    }
  }
}

/* ----------------------------------------------------------- one path ---- */
typedef struct {
  const oracle_system* sys;
  int sys_index;
  int64_t path;          /* path id within its system */
  int64_t n_therm, n_meas;
  uint32_t k0, k1;
  int init_mode, order_mode;
  double* rec;           /* NREC doubles */
  double* spins_out;     /* 3N doubles or NULL */
} path_job;

static void run_path(const path_job* jb) {
  const oracle_system* sy = jb->sys;
  const int lat = sy->lattice, L = sy->L;
  const int64_t N = n_sites(lat, L);
  const double beta = 1.0 / sy->T, J = sy->J, hf = sy->h;
  const uint32_t c2 = (uint32_t)jb->path;
  const uint32_t sys_hi = (uint32_t)jb->sys_index << 8;
  double* s = (double*)malloc(sizeof(double) * 3 * N);
  uint32_t r[4];

  init_state(N, c2, sys_hi, jb->k0, jb->k1, jb->init_mode, s);

  double acc[NREC];
  memset(acc, 0, sizeof(acc));
  int64_t accepted = 0;
  const int64_t S = jb->n_therm + jb->n_meas;

  for (int64_t sw = 0; sw < S; ++sw) {
    /* one lattice sweep = N Metropolis attempts */
    if (jb->order_mode == OR_ORDER_RANDOM) {
      /* the paper's order: N sites drawn at random (Sec. 2.2).  Attempt a
       * of the sweep takes one counter (a, sweep, path, 2 | sys<<8): the site
       * is the cell of width 1/N holding u(r[3]), i = floor((2 r3 + 1) N / 2^33)
       * in exact integer arithmetic, and r[0..2] drive the move as in the
       * checkerboard order. */
      for (int64_t a = 0; a < N; ++a) {
        oracle_philox((uint32_t)a, (uint32_t)sw, c2, OR_TAG_SITE | sys_hi, jb->k0, jb->k1, r);
        const int64_t i = (int64_t)((((uint64_t)r[3] * 2u + 1u) * (uint64_t)N) >> 33);
        accepted += metropolis(lat, L, J, hf, beta, s, i, r);
      }
    } else {
      /* checkerboard: every colour-0 site, then every colour-1 site */
      for (int c = 0; c < 2; ++c) {
        for (int64_t i = 0; i < N; ++i) {
          if (colour(lat, L, i) != c) continue;
          oracle_philox((uint32_t)i, (uint32_t)sw, c2, OR_TAG_UPDATE | sys_hi, jb->k0, jb->k1, r);
          accepted += metropolis(lat, L, J, hf, beta, s, i, r);
        }
      }
    }

    if (sw >= jb->n_therm) {
      /* per-site observables of the current state (Sec. 2.2) */
      double mx = 0.0, my = 0.0, mz = 0.0;
      for (int64_t i = 0; i < N; ++i) {
        mx += s[3 * i + 0]; my += s[3 * i + 1]; mz += s[3 * i + 2];
      }
      mx /= (double)N; my /= (double)N; mz /= (double)N;
      double e = oracle_energy(lat, L, J, hf, s) / (double)N;
      double m = sqrt(mx * mx + my * my + mz * mz);
      acc[R_E] += e;
      acc[R_E2] += e * e;
      acc[R_M] += m;
      acc[R_M2] += m * m;
      acc[R_M4] += m * m * m * m;
      acc[R_MX] += mx;
      acc[R_MY] += my;
      acc[R_MZ] += mz;
      acc[R_MZ2] += mz * mz;
      acc[R_AMZ] += fabs(mz);
      acc[R_EM] += e * m;
      acc[R_EMZ] += e * mz;
      acc[R_MMZ] += m * mz;
      if (sw == S - 1) {
        acc[R_FMX] = mx; acc[R_FMY] = my; acc[R_FMZ] = mz; acc[R_FE] = e;
      }
    }
  }

  double* out = jb->rec;
  for (int k = R_E; k <= R_MMZ; ++k) out[k] = acc[k] / (double)jb->n_meas;
  out[R_FMX] = acc[R_FMX]; out[R_FMY] = acc[R_FMY];
  out[R_FMZ] = acc[R_FMZ]; out[R_FE] = acc[R_FE];
  out[R_ACC] = (double)accepted / ((double)S * (double)N);
  double worst = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double n2 = s[3 * i] * s[3 * i] + s[3 * i + 1] * s[3 * i + 1] + s[3 * i + 2] * s[3 * i + 2];
    double d = fabs(sqrt(n2) - 1.0);
    if (d > worst) worst = d;
  }
  out[R_NORM] = worst;
  out[R_SPARE] = 0.0;
  if (jb->spins_out) memcpy(jb->spins_out, s, sizeof(double) * 3 * N);
  free(s);
}

/* ------------------------------------------------------ 2D Ising path ----
 * Appendix A runs the same multipath scheme on the square-lattice Ising model.
 * Readings (the appendix gives no formulas):
 *   - H = -J sum_bonds s_i s_j - h sum_i s_i, s_i = +-1, periodic L x L, L even;
 *     site i = x + L y, colour (x + y) mod 2, neighbours +x, -x, +y, -y;
 *   - random start: s_i = +1 when the top bit of word 0 of the init counter
 *     (i, 0, path, 1 | sys<<8) is clear, else -1; ordered start: all +1;
 *   - a sweep flips-tests every colour-0 site, then every colour-1 site;
 *     dE = 2 s_i (J sum_nb s_j + h), accept when dE <= 0, else iff
 *     u < exp(-beta dE) with u = (r + 1/2) 2^-32;
 *   - the word r of the colour-c site in row y with x/2 = hx is word y mod 4
 *     of Philox(hx + (L/2) (y / 4), sweep, path, (4 + c) | sys<<8): one call
 *     serves the four sites of one colour in rows 4j .. 4j+3 at the same x/2;
 *   - per sweep: e = H / N and m = sum s_i / N; the record keeps the
 *     Heisenberg layout with m_x = m_y = 0 and m_z = m. */
static void run_path_ising(const path_job* jb) {
  const oracle_system* sy = jb->sys;
  const int L = sy->L;
  const int64_t N = (int64_t)L * L;
  const double beta = 1.0 / sy->T, J = sy->J, hf = sy->h;
  const uint32_t c2 = (uint32_t)jb->path;
  const uint32_t sys_hi = (uint32_t)jb->sys_index << 8;
  int* s = (int*)malloc(sizeof(int) * N);
  uint32_t r[4];
  for (int64_t i = 0; i < N; ++i) {
    oracle_philox((uint32_t)i, 0u, c2, OR_TAG_INIT | sys_hi, jb->k0, jb->k1, r);
    s[i] = (jb->init_mode == OR_INIT_ORDERED) ? 1 : ((r[0] >> 31) ? -1 : 1);
  }
  double acc[NREC];
  memset(acc, 0, sizeof(acc));
  int64_t accepted = 0;
  const int64_t S = jb->n_therm + jb->n_meas;
  for (int64_t sw = 0; sw < S; ++sw) {
    for (int c = 0; c < 2; ++c) {
      for (int64_t i = 0; i < N; ++i) {
        const int64_t x = i % L, y = i / L;
        if (((x + y) & 1) != c) continue;
        const int64_t hx = x >> 1;
        oracle_philox((uint32_t)(hx + (L / 2) * (y >> 2)), (uint32_t)sw, c2,
                      (OR_TAG_ISING + (uint32_t)c) | sys_hi, jb->k0, jb->k1, r);
        const int64_t nb[4] = {(x + 1) % L + L * y, (x + L - 1) % L + L * y,
                               x + L * ((y + 1) % L), x + L * ((y + L - 1) % L)};
        const int hloc = s[nb[0]] + s[nb[1]] + s[nb[2]] + s[nb[3]];
        const double dE = 2.0 * (double)s[i] * (J * (double)hloc + hf);
        if (dE <= 0.0 || u01(r[y & 3]) < exp(-beta * dE)) {
          s[i] = -s[i];
          ++accepted;
        }
      }
    }
    if (sw >= jb->n_therm) {
      int64_t bonds = 0, msum = 0;
      for (int64_t i = 0; i < N; ++i) {
        const int64_t x = i % L, y = i / L;
        bonds += (int64_t)s[i] * (s[(x + 1) % L + L * y] + s[x + L * ((y + 1) % L)]);
        msum += s[i];
      }
      const double e = (-J * (double)bonds - hf * (double)msum) / (double)N;
      const double mz = (double)msum / (double)N;
      const double m = fabs(mz);
      acc[R_E] += e;
      acc[R_E2] += e * e;
      acc[R_M] += m;
      acc[R_M2] += m * m;
      acc[R_M4] += m * m * m * m;
      acc[R_MZ] += mz;
      acc[R_MZ2] += mz * mz;
      acc[R_AMZ] += m;
      acc[R_EM] += e * m;
      acc[R_EMZ] += e * mz;
      acc[R_MMZ] += m * mz;
      if (sw == S - 1) {
        acc[R_FMZ] = mz; acc[R_FE] = e;
      }
    }
  }
  double* out = jb->rec;
  for (int k = R_E; k <= R_MMZ; ++k) out[k] = acc[k] / (double)jb->n_meas;
  out[R_FMX] = 0.0; out[R_FMY] = 0.0;
  out[R_FMZ] = acc[R_FMZ]; out[R_FE] = acc[R_FE];
  out[R_ACC] = (double)accepted / ((double)S * (double)N);
  out[R_NORM] = 0.0;
  out[R_SPARE] = 0.0;
  if (jb->spins_out) {
    for (int64_t i = 0; i < N; ++i) {
      jb->spins_out[3 * i + 0] = 0.0;
      jb->spins_out[3 * i + 1] = 0.0;
      jb->spins_out[3 * i + 2] = (double)s[i];
    }
  }
  free(s);
}

/* ------------------------------------------------------------ threads ---- */
typedef struct {
  path_job* jobs;
  int64_t n_jobs;
  int64_t next;
  pthread_mutex_t mu;
} job_queue;

static void* worker(void* arg) {
  job_queue* q = (job_queue*)arg;
  for (;;) {
    pthread_mutex_lock(&q->mu);
    int64_t j = q->next++;
    pthread_mutex_unlock(&q->mu);
    if (j >= q->n_jobs) return NULL;
    if (q->jobs[j].sys->lattice == OR_ISING)
      run_path_ising(&q->jobs[j]);
    else
      run_path(&q->jobs[j]);
  }
}

int oracle_nrec(void) { return NREC; }

/* Runs every requested path.  records: sum(path_count) x NREC doubles, in
 * system order then path order.  spins_out (optional): 3N doubles per path in
 * the same order (site-major, x y z).  Returns 0, or -1 on bad arguments. */
int oracle_run(const oracle_system* sys, int n_sys, int64_t n_therm, int64_t n_meas,
               uint64_t seed, int init_mode, int order_mode, int n_threads,
               double* records, double* spins_out) {
  if (!sys || n_sys <= 0 || n_therm < 0 || n_meas < 1 || !records) return -1;
  int64_t total = 0;
  for (int k = 0; k < n_sys; ++k) {
    const oracle_system* sy = &sys[k];
    if (sy->lattice != OR_SC && sy->lattice != OR_CHAIN && sy->lattice != OR_ISING) return -1;
    if (sy->lattice == OR_ISING && ((sy->L & 1) || order_mode != OR_ORDER_CHECKER)) return -1;
    if (sy->L < 2 || !(sy->T > 0.0) || sy->n_paths <= 0) return -1;
    if (sy->lattice == OR_SC && (sy->L & 1) && order_mode == OR_ORDER_CHECKER) return -1;
    if (sy->path_begin < 0 || sy->path_count < 0 ||
        sy->path_begin + sy->path_count > sy->n_paths)
      return -1;
    total += sy->path_count;
  }
  path_job* jobs = (path_job*)calloc((size_t)(total > 0 ? total : 1), sizeof(path_job));
  int64_t j = 0, spin_off = 0;
  for (int k = 0; k < n_sys; ++k) {
    int64_t N = n_sites(sys[k].lattice, sys[k].L);
    for (int64_t p = 0; p < sys[k].path_count; ++p, ++j) {
      jobs[j].sys = &sys[k];
      jobs[j].sys_index = k;
      jobs[j].path = sys[k].path_begin + p;
      jobs[j].n_therm = n_therm;
      jobs[j].n_meas = n_meas;
      jobs[j].k0 = (uint32_t)(seed & 0xffffffffu);
      jobs[j].k1 = (uint32_t)(seed >> 32);
      /* Sec. 4's convergence check: with OR_TWO_START the first ceil(P/2)
       * paths start from init_mode, the other floor(P/2) from the ordered
       * state, and the two halves are averaged separately. */
      jobs[j].init_mode = init_mode & 0xff;
      if ((init_mode & OR_TWO_START) && jobs[j].path >= sys[k].n_paths - sys[k].n_paths / 2)
        jobs[j].init_mode = OR_INIT_ORDERED;
      jobs[j].order_mode = order_mode;
      jobs[j].rec = records + j * NREC;
      jobs[j].spins_out = spins_out ? spins_out + spin_off : NULL;
      spin_off += 3 * N;
    }
  }
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 1024) n_threads = 1024;
  job_queue q;
  q.jobs = jobs; q.n_jobs = total; q.next = 0;
  pthread_mutex_init(&q.mu, NULL);
  pthread_t th[1024];
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &q);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&q.mu);
  free(jobs);
  return 0;
}

/* Trial direction from the update stream of (site, sweep, path, system):
 * exposes the trial move for statistical pins on the proposal. */
void oracle_trial(uint32_t site, uint32_t sweep, uint32_t path, uint32_t sys_index,
                  uint64_t seed, double out[3]) {
  uint32_t r[4];
  oracle_philox(site, sweep, path, OR_TAG_UPDATE | (sys_index << 8),
                (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), r);
  sphere_point(u01(r[0]), u01(r[1]), out);
}

/* Initial state of one path (3N doubles, site-major). */
int oracle_init(int lattice, int L, uint32_t path, uint32_t sys_index, uint64_t seed,
                int init_mode, double* out) {
  if ((lattice != OR_SC && lattice != OR_CHAIN) || L < 1 || !out) return -1;
  init_state(n_sites(lattice, L), path, sys_index << 8, (uint32_t)(seed & 0xffffffffu),
             (uint32_t)(seed >> 32), init_mode, out);
  return 0;
}
