/*
 * mp.h -- C ABI of the GB300 multipath Metropolis library for the classical
 * O(3) Heisenberg model (Rakic, Radosevic, Mali, Stricevic, Petric,
 * "Multipath Metropolis Simulation of Classical Heisenberg Model").
 *
 * The method (Sec. 2.2): many mutually independent Metropolis random walks
 * ("simulation paths") of one lattice at one temperature, each started from a
 * random state, thermalised by lattice sweeps and then measured; the per-path
 * outputs {M^x, M^y, M^z, H} (per lattice site) are averaged over paths,
 * Eq. (MCAV), into ensemble estimates with standard errors.
 *
 * Model (Sec. 2.1): H = -(J/2) sum_n sum_lambda S_n . S_{n+lambda} - h sum_n S^z_n,
 * Eq. (1) plus a Zeeman term (h = 0 is the paper's model), unit spins of Eq. (2),
 * on a periodic simple-cubic lattice of N = L^3 sites (L even, at most 1024;
 * L <= 26 in FP32 and L <= 20 in FP64 run with the lattice in shared memory,
 * FP32 L = 32 in the shared memory of a two-CTA cluster, larger lattices are
 * streamed from HBM while their half-plane ring fits in shared memory: L <= 64
 * in FP32, L <= 44 in FP64, and updated in place in HBM beyond that) or an
 * open chain of N = L spins.
 *
 * Conventions shared by every call:
 *   - Every function returns an int status (MP_OK or a negative MP_E* code),
 *     except mp_destroy and the string helpers.  On error nothing observable
 *     changes except the handle's last-error text (mp_last_error).
 *   - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *     pointers are CUDA global memory on the handle's device.
 *   - A handle is not thread-safe: use one handle per host thread.
 *   - All GPU work of a handle is issued on its stream (mp_config.stream);
 *     calls that return host data synchronise that stream first.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low 32
 *     bits, seed high 32 bits), counter = (site, sweep, path id within its
 *     system, tag | system index << 8), tag 0 = update, 1 = initial state.
 *     Results are therefore a pure function of (config, seed), independent of
 *     launch shape and GPU.
 */
#ifndef MP_H
#define MP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */
#define MP_OK 0
#define MP_EINVAL (-1)     /* bad argument (see each call) */
#define MP_ENOMEM (-2)     /* the allocator returned NULL */
#define MP_ECUDA (-3)      /* a CUDA runtime call failed; see mp_last_error */
#define MP_ESTATE (-4)     /* call out of order, e.g. estimates before a run */
#define MP_ECANCELED (-5)  /* mp_cancel stopped the run before it finished */
#define MP_ETIMEOUT (-6)   /* a bounded wait in a kernel gave up (a bulk copy of
                              the streamed path did not arrive within ~2 s); the
                              run's results are invalid, the context stays usable */

/* ---------------------------------------------------------------- enums --- */
#define MP_LATTICE_SC 0    /* periodic simple cubic, N = L^3, L even */
#define MP_LATTICE_CHAIN 1 /* open chain, N = L >= 2 */
#define MP_LATTICE_ISING 2 /* Appendix A: periodic L x L square lattice of Ising
                              spins s = +-1, N = L^2, L even in 2..MP_ISING_MAX_L;
                              H = -J sum_bonds s_i s_j - h sum_i s_i.  A batch
                              is either all Ising or all Heisenberg; precision
                              and init_mode ANGLES do not apply (the random
                              start draws each sign with probability 1/2).
                              Records use the Heisenberg layout with
                              m_x = m_y = 0, m_z = m; spins (mp_spins) are
                              (0, 0, s) per site. */
#define MP_ISING_MAX_L 256

#define MP_FP32 0 /* FP32 spins, dE and Boltzmann factor; FP64 accumulators */
#define MP_FP64 1 /* FP64 throughout (the plain FP64 GPU form) */

#define MP_INIT_SPHERE 0  /* uniform on the sphere (Sec. 4, "uniform state") */
#define MP_INIT_ANGLES 1  /* theta, phi each uniform (Sec. 2.2 "both angles") */
#define MP_INIT_ORDERED 2 /* all spins along +z (Sec. 5, ordered start) */

#define MP_FLAG_GRAPH 1u      /* capture each run in a CUDA graph and replay it */
#define MP_FLAG_KEEP_SPINS 2u /* keep every path's final spins (mp_spins) */
#define MP_FLAG_STREAM 4u     /* stream every simple-cubic lattice from HBM, even
                                 those that fit in shared memory (lattices too
                                 large for shared memory are always streamed) */
#define MP_FLAG_AUTOTUNE 8u   /* at create, time a few threads-per-path layouts of
                                 each system in the batch's own kernel (one
                                 wave of its work items, ~2e8 attempts each)
                                 and keep the fastest; ignored when
                                 threads_per_path is set.  The choice is
                                 remembered for the life of the process: a
                                 later create of a batch of the same shape
                                 (device, precision, init mode, cta_threads,
                                 and per system lattice, L, n_paths) on the
                                 same device takes it without timing */
#define MP_FLAG_TWO_START 16u /* Sec. 4's convergence check: in every system the
                                 first ceil(P/2) paths start from init_mode, the
                                 other floor(P/2) from the ordered state; the
                                 estimates report both halves (e_a, e_b, ...) */
#define MP_FLAG_RANDOM_SITE 32u /* the paper's literal sweep order (Sec. 2.2): a
                                 sweep is N attempts at sites drawn at random
                                 (attempt a of sweep s: counter (a, s, path,
                                 2 | sys<<8), site floor((2 r3 + 1) N / 2^33),
                                 move from r0..r2).  One thread per path, spins
                                 in HBM; simple-cubic and chain systems only;
                                 mp_run_sweeps, mp_checkpoint and mp_restore
                                 return MP_EINVAL */
#define MP_FLAG_TEST_STALL 0x100u /* failure injection for tests: streamed paths
                                     never issue their first bulk copy, so the
                                     kernel's bounded wait runs out (about 2 s)
                                     and mp_estimates returns MP_ETIMEOUT */
#define MP_FLAG_DEVICE_UNITS 0x200u /* for tests: make no column-walk unit tables;
                                       the shared-memory walk derives each unit
                                       on the device instead (the same units and
                                       results, more instructions per unit) */

/* ------------------------------------------------------------- records ---
 * Per-path record: MP_NREC doubles per path.  Fields 0..12 are means over the
 * path's n_meas measurement sweeps of per-site observables of the state after
 * each sweep: e = H/N (energy per site, Eq. 1 plus Zeeman term) and
 * m = (1/N) sum_n S_n (Sec. 2.2).  Fields 13..16 are the state after the last
 * sweep (the paper's per-path output {M^x, M^y, M^z, H}).  n_meas = 1 gives
 * exactly the paper's single final-state output. */
enum {
  MP_R_E = 0,   /* <e> */
  MP_R_E2,      /* <e^2> */
  MP_R_M,       /* <|m|> */
  MP_R_M2,      /* <|m|^2> */
  MP_R_M4,      /* <|m|^4> */
  MP_R_MX,      /* <m_x> */
  MP_R_MY,      /* <m_y> */
  MP_R_MZ,      /* <m_z> */
  MP_R_MZ2,     /* <m_z^2> */
  MP_R_AMZ,     /* <|m_z|> */
  MP_R_EM,      /* <e |m|> */
  MP_R_EMZ,     /* <e m_z> */
  MP_R_MMZ,     /* <|m| m_z> */
  MP_R_FMX,     /* final m_x */
  MP_R_FMY,     /* final m_y */
  MP_R_FMZ,     /* final m_z */
  MP_R_FE,      /* final e */
  MP_R_ACC,     /* accepted / attempted moves over all sweeps */
  MP_R_NORM,    /* max over sites of | |S| - 1 | in the final state */
  MP_R_SPARE,
  MP_NREC
};

/* ----------------------------------------------------------- estimates ---
 * Ensemble estimates of one system, all doubles.  <A> is the mean over paths
 * of the per-path means, Eq. (MCAV); *_se is its standard error
 * (sample standard deviation over paths / sqrt(paths)).
 *   chi      = (N/T) (<|m|^2> - <|m|>^2)                     Eq. (cv), left
 *   cv       = (N/T^2) (<e^2> - <e>^2)                       Eq. (cv), right
 *   binder   = 1 - <|m|^4> / (3 <|m|^2>^2)                   Eq. (kum)
 *   dX_dbeta = -N (<X e> - <X><e>)       (fluctuation formula, X in {e,|m|,m_z})
 *   dX_dh    = beta N (<X m_z> - <X><m_z>) + <dX/dh>, where only X = e has
 *              an explicit field term: de/dh = -m_z, so de_dh carries -<m_z>
 *   cv_m     = se(<|m|>) / <|m|>                             Eq. (eq:cv)
 *   r_*      = 1 - ||R||^2 / ((P-1) sigma^2) of the normal Q-Q line fit of the
 *              per-path values, plotting positions (i - 1/2)/P,
 *              Eq. (dist-coefficient); NaN when P < 3.  Up to MP_R_MAX_PATHS
 *              paths the values are sorted in shared memory; a handle with a
 *              larger system sorts in a device buffer of 2 P doubles per
 *              system, allocated at create.
 * SEs of derived quantities are delete-one jackknife over paths. */
#define MP_R_MAX_PATHS 16384

typedef struct {
  double n_paths, N, T, n_meas;
  double e, e_se, e2, e2_se;
  double m, m_se, m2, m2_se, m4, m4_se;
  double mx, mx_se, my, my_se, mz, mz_se;
  double mz2, mz2_se, amz, amz_se;
  double acc, acc_se;
  double chi, chi_se, cv, cv_se, binder, binder_se;
  double de_dbeta, de_dbeta_se, dm_dbeta, dm_dbeta_se, dmz_dbeta, dmz_dbeta_se;
  double de_dh, de_dh_se, dm_dh, dm_dh_se, dmz_dh, dmz_dh_se;
  double cv_m;
  double r_e, r_m, r_mx, r_my, r_mz, r_amz;
  double attempts; /* N x paths x (n_therm + n_meas) */
  double norm_max; /* max over paths of MP_R_NORM */
  /* The first ceil(P/2) paths (a) and the other floor(P/2) (b) averaged
   * separately; with MP_FLAG_TWO_START they started from init_mode and from
   * the ordered state (Sec. 4).  start_z = max over X in {e, |m|} of
   * |X_a - X_b| / sqrt(X_a_se^2 + X_b_se^2), skipping an undefined 0/0. */
  double e_a, e_a_se, e_b, e_b_se, m_a, m_a_se, m_b, m_b_se, start_z;
  /* Device time of the run these estimates come from, in seconds: the sweep
   * kernel and the reduction kernel, from CUDA events on the handle's stream
   * (filled in by mp_estimates; NaN from mp_run_noalloc, which records no
   * events). */
  double elapsed_s;
  double reserved[1];
} mp_estimates_t; /* 64 doubles */

#define MP_NEST 64

/* --------------------------------------------------------------- config -- */
typedef struct {
  int32_t lattice; /* MP_LATTICE_* */
  int32_t L;       /* linear size (SC) or number of spins (chain) */
  double T;        /* temperature, k_B = 1 (Sec. 2.1 fixes J = 1 as the scale) */
  double J;        /* exchange; J > 0 ferro, J < 0 antiferro (Sec. 2.1) */
  double h;        /* field along +z (not in the paper; 0 reproduces it) */
  int64_t n_paths; /* independent paths of this system, >= 1 */
  int64_t path_begin; /* path id of the first path: path k of the system draws
                         the random numbers of path id path_begin + k, so
                         processes that split one ensemble run disjoint ranges
                         with the same seed; 0 for a whole ensemble.
                         path_begin + n_paths <= 2^32.  MP_FLAG_TWO_START
                         halves the local range 0 .. n_paths-1 */
} mp_system;

/* Device-memory allocator hooks.  alloc must return device memory of at least
 * `bytes` bytes aligned to 256 bytes, or NULL; free releases it.  Both are
 * called only from mp_create_ex / mp_destroy on the calling thread.  When
 * alloc_fn is NULL the library uses cudaMalloc / cudaFree. */
typedef void* (*mp_alloc_fn)(void* ctx, size_t bytes);
typedef void (*mp_free_fn)(void* ctx, void* ptr);

typedef struct {
  int32_t precision;     /* MP_FP32 or MP_FP64 */
  int32_t init_mode;     /* MP_INIT_* */
  int32_t n_systems;     /* >= 1 */
  uint32_t flags;        /* MP_FLAG_* */
  const mp_system* systems; /* host array of n_systems, copied at create */
  int64_t n_therm;       /* thermalisation sweeps, >= 0 */
  int64_t n_meas;        /* measurement sweeps, >= 1 */
  uint64_t seed;         /* Philox key */
  void* stream;          /* cudaStream_t for all work; NULL = a non-blocking
                            stream the handle creates and owns */
  mp_alloc_fn alloc_fn;  /* optional */
  mp_free_fn free_fn;    /* required when alloc_fn is set */
  void* alloc_ctx;
  int32_t cta_threads;   /* threads per CTA: 0 = planner default, else 128..1024 */
  int32_t threads_per_path; /* 0 = planner default, else a multiple of 32 */
} mp_config;

typedef struct mp_state* mp_handle;

/* ----------------------------------------------------------------- calls -- */

/* Create a handle for one system: periodic simple-cubic lattice of L^3 spins
 * at temperature T with n_paths independent paths of n_therm thermalisation
 * and n_meas measurement sweeps (Sec. 2.2: "a particular lattice size at a
 * particular temperature ... a certain number of simulation paths").  FP32
 * form, uniform-on-sphere start, CUDA-graph replay, current device, a stream
 * of the handle's own.  *out receives the handle (NULL on error).
 * Errors: MP_EINVAL (out NULL, L odd or outside the supported sizes, T <= 0,
 * n_paths < 1, n_therm < 0, n_meas < 1, path ids beyond 2^32, sweeps beyond
 * 2^32), MP_ENOMEM, MP_ECUDA. */
int mp_create(int L, double T, double J, double h, int64_t n_paths, int64_t n_therm,
              int64_t n_meas, uint64_t seed, mp_handle* out);

/* Create a handle for a batch of systems (uneven lattice sizes allowed) that
 * run together in one persistent launch per run.  cfg and cfg->systems are
 * read during the call only.  Device buffers (records, estimates, work
 * table) are allocated here through cfg->alloc_fn and owned by the handle.
 * Errors: as mp_create, plus MP_EINVAL for n_systems < 1 or > 65535, unknown
 * lattice/precision/init mode, a lattice too large for the precision's
 * shared-memory kernel, alloc_fn without free_fn. */
int mp_create_ex(const mp_config* cfg, mp_handle* out);

/* Run every path of every system from its initial state: n_therm + n_meas
 * checkerboard sweeps with fused measurement, then the cross-path reduction.
 * Asynchronous on the handle's stream; re-running repeats the same
 * computation (use mp_set_seed for a new ensemble).
 * Errors: MP_EINVAL (h NULL), MP_ECUDA (launch failure). */
int mp_run(mp_handle h);

/* Change the Philox key used by the next mp_run.  No GPU work. */
int mp_set_seed(mp_handle h, uint64_t seed);

/* Copy the estimates of system `system` (0-based, in mp_config order) into
 * the caller's *out.  Synchronises the stream.
 * Errors: MP_EINVAL (bad index, out NULL), MP_ESTATE (no run yet),
 * MP_ECUDA (an asynchronous error surfaced). */
int mp_estimates(mp_handle h, int system, mp_estimates_t* out);

/* Copy the per-path records of one system, MP_NREC doubles per path, path
 * order, into host_out (capacity `cap` doubles, must be >= n_paths*MP_NREC).
 * Synchronises.  Errors: MP_EINVAL, MP_ESTATE, MP_ECUDA. */
int mp_paths(mp_handle h, int system, double* host_out, int64_t cap);

/* Device pointers to the handle's per-path records (all systems, system
 * order, MP_NREC doubles per path) and estimates (MP_NEST doubles per system).
 * Owned by the handle; valid until mp_destroy; contents valid once the
 * stream has completed a run.  Either output may be NULL. */
int mp_device_buffers(mp_handle h, double** d_records, double** d_estimates);

/* Copy the final spins of one path (3N doubles, site-major x,y,z, site index
 * x + L(y + Lz)) into host_out (capacity cap doubles).  Requires
 * MP_FLAG_KEEP_SPINS.  Synchronises.  Errors: MP_EINVAL, MP_ESTATE. */
int mp_spins(mp_handle h, int system, int64_t path, double* host_out, int64_t cap);

/* Fluctuation-formula backward of the per-site observables (<e>, <|m|>) of
 * every system: for each system s,
 *   d_grad_beta[s] = g_e[s] d<e>/dbeta + g_m[s] d<|m|>/dbeta
 *   d_grad_h[s]    = g_e[s] d<e>/dh    + g_m[s] d<|m|>/dh
 * with d/dbeta = -N cov(., e), d/dh = beta N cov(., m_z) over the per-path
 * pooled moments (the estimators of C_V and chi, Eq. (cv)), plus -<m_z> in
 * d<e>/dh from the field term of e itself.  All four arrays
 * are device memory of n_systems doubles, owned by the caller; the kernel is
 * queued on the handle's stream after the last run.
 * Errors: MP_EINVAL (NULL pointer), MP_ESTATE (no run yet), MP_ECUDA. */
int mp_backward(mp_handle h, const double* d_g_e, const double* d_g_m,
                double* d_grad_beta, double* d_grad_h);

/* Device-side durations of the last run's sweep kernel and reduction kernel,
 * from CUDA events recorded on the handle's stream.  Synchronises.
 * Errors: MP_ESTATE (no run yet), MP_ECUDA. */
int mp_timing(mp_handle h, double* sweep_ms, double* reduce_ms);

/* Launch shape chosen for the handle: CTA threads, CTAs in the persistent
 * grid, dynamic shared memory bytes per CTA, work items.  Any output may be
 * NULL. */
int mp_plan(mp_handle h, int* cta_threads, int* grid, int* smem_bytes, int* n_items);

/* Bytes of the plan's tables (systems, work items, offsets, Ising thresholds,
 * column-walk units) that the handle last copied from host to device: once
 * when it is created, for the plan its runs then use.  Errors: MP_EINVAL
 * (NULL handle or output). */
int mp_upload_bytes(mp_handle h, int64_t* bytes);

/* Resumable runs.  mp_run_sweeps advances every path of every system by
 * n_sweeps sweeps of its schedule (n_therm thermalisation sweeps, then n_meas
 * measurement sweeps) from its saved state -- the initial state on the first
 * call -- and saves the state again (per path: FP64 accumulators, acceptance
 * count, spins; kept in device memory owned by the handle, allocated on the
 * first call).  Records and estimates then cover the measurement sweeps done
 * so far.  Splitting a schedule into several calls gives the same
 * trajectories as one call (the random numbers depend only on seed, system,
 * path, sweep and site).  Synchronises; the progress advances only when the
 * call succeeds.  Independent of mp_run, which always runs the whole schedule.
 * Errors: MP_EINVAL (n_sweeps < 1), MP_ESTATE (schedule already complete),
 * MP_ENOMEM, MP_ECANCELED (mp_cancel during the call; state unchanged),
 * MP_ETIMEOUT, MP_ECUDA. */
int mp_run_sweeps(mp_handle h, int64_t n_sweeps);

/* Sweeps of the schedule done by mp_run_sweeps so far (or restored). */
int mp_progress(mp_handle h, int64_t* sweeps_done);

/* Checkpoint of the resumable state.  With buf NULL, *nbytes receives the
 * size; otherwise buf (caller-owned host memory of *nbytes bytes) receives a
 * versioned header and the state, and *nbytes the bytes written.  The
 * checkpoint is valid for a handle of the same configuration (systems,
 * precision, init mode, seed, schedule, lattice modes).  Synchronises.
 * Errors: MP_EINVAL (NULL, buffer too small), MP_ESTATE (no mp_run_sweeps yet). */
int mp_checkpoint(mp_handle h, void* buf, size_t* nbytes);

/* Load a checkpoint written by mp_checkpoint (host memory, read during the
 * call) into a handle of the same configuration; the next mp_run_sweeps
 * continues from it.  Errors: MP_EINVAL (not a checkpoint, other
 * configuration, wrong size), MP_ENOMEM, MP_ECUDA. */
int mp_restore(mp_handle h, const void* buf, size_t nbytes);

/* Ask the handle's running or next-started kernels to stop: they poll a
 * host-mapped flag every 16 sweeps, stop at a sweep boundary and write no
 * record; mp_estimates / mp_paths then return MP_ECANCELED and mp_run_sweeps
 * leaves the saved state unchanged.  The flag is cleared when the next run
 * starts.  The one call that may be made from another host thread while a
 * run is in flight. */
int mp_cancel(mp_handle h);

/* Launch shape of one system: threads per path, paths per CTA, and where
 * its lattice lives during a run: 0 in one CTA's shared memory, 1 streamed
 * from HBM through shared-memory half-plane buffers, 2 split over the shared
 * memory of the two CTAs of a cluster (FP32 simple cubic L = 32: each CTA
 * holds half of the z-planes, one path per cluster, threads_per_path then
 * counts one CTA), 3 updated in place in HBM (lattices whose half-plane ring
 * does not fit: FP64 L >= 46, FP32 L >= 66).  Any output may be NULL.
 * Errors: MP_EINVAL (bad index). */
int mp_system_plan(mp_handle h, int system, int* threads_per_path, int* paths_per_cta,
                   int* streamed_from_hbm);

/* Ensemble estimates of per-path records the caller holds: the reduction
 * kernel of mp_run (Sec. 2.2: Eq. MCAV, Eq. cv, Eq. kum, Eq. eq:cv and the
 * distribution coefficient of Sec. 3) on d_records, MP_NREC doubles per path,
 * the systems' paths one after another in `systems` order (device memory,
 * caller-owned, read only), written to d_estimates, MP_NEST doubles per
 * system (device memory, caller-owned; elapsed_s is NaN).  n_therm and n_meas
 * are the schedule the records come from (they enter n_meas and attempts).
 * For processes that each ran part of one ensemble (disjoint path_begin
 * ranges of the same systems and seed): gather their records in path order
 * and reduce them here to obtain exactly the estimates of one process
 * running every path.  Allocates and frees a small device table (and, for
 * systems of more than MP_R_MAX_PATHS paths, 2 x paths doubles of sort
 * space) and synchronises `stream` (cudaStream_t; NULL = legacy default).
 * Errors: MP_EINVAL (NULL pointer, bad system), MP_ENOMEM, MP_ECUDA; the text
 * is mp_last_error(NULL). */
int mp_reduce(const mp_system* systems, int n_systems, int64_t n_therm, int64_t n_meas,
              const double* d_records, double* d_estimates, void* stream);

/* Philox4x32-10 of n counters: d_ctr holds 4n uint32 words (c0 c1 c2 c3 per
 * counter), d_out receives 4n words.  Device pointers, caller-owned; queued
 * on `stream` (cudaStream_t, NULL = legacy default).  The same device function
 * the sweep kernels use.  Errors: MP_EINVAL (n < 0, NULL with n > 0), MP_ECUDA. */
int mp_philox(const uint32_t* d_ctr, int64_t n, uint64_t seed, uint32_t* d_out, void* stream);

/* Allocation-free run, for callers that cannot allocate device memory:
 * code inside a host framework that owns every device allocation (a fixed
 * pool or arena), code that must not grow the device heap after start-up, or
 * a plugin whose host forbids allocator calls.  The paper has no counterpart;
 * the call exists for those callers.
 *
 * It runs the same sweep and reduction kernels as mp_run for the batch
 * `systems` (host array of n_systems, read during the call) in `precision`
 * (MP_FP32 or MP_FP64) with uniform-on-sphere starts, and writes MP_NEST
 * doubles of estimates per system (the mp_estimates_t layout) to d_estimates
 * (device memory of n_systems * MP_NEST doubles, owned by the caller), all
 * queued on `stream` (cudaStream_t; NULL = legacy default stream).  It calls
 * no cudaMalloc, cudaFree or other allocating routine: its scratch (per-path
 * records, work queue, device copies of the tables) is one static __device__
 * array of about 3.4 MB that every GPU loading the library holds until the
 * process exits.  Limits: at most MP_NOALLOC_MAX_PATHS paths in total and
 * MP_NOALLOC_MAX_SYSTEMS systems; larger batches return MP_EINVAL before any
 * GPU work.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  All calls share the
 * one array and it keeps the last call's contents (the work counter is
 * cleared at the start of each call): calls whose GPU work overlaps, on
 * different streams or different host threads, race on it.  Errors: MP_EINVAL (NULL pointer, bad sizes,
 * unsupported lattice), MP_ECUDA (device error). */
#define MP_NOALLOC_MAX_PATHS 16384
#define MP_NOALLOC_MAX_SYSTEMS 64
int mp_run_noalloc(const mp_system* systems, int n_systems, int precision, int64_t n_therm,
                   int64_t n_meas, uint64_t seed, double* d_estimates, void* stream);

/* Release every device buffer, event and graph of the handle (after
 * synchronising its stream).  NULL is a no-op. */
void mp_destroy(mp_handle h);

/* Text of the last error on the handle ("" if none); valid until the next
 * call on the handle.  NULL handle: the last error of a failed create on this
 * thread. */
const char* mp_last_error(mp_handle h);

/* Name of a status code. */
const char* mp_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* MP_H */
