/*
 * fmm_vortex.h -- C ABI of the GB300 (sm_103a) FMM for vortex particles.
 *
 * One call evaluates, for N Gaussian vortex blobs, the regularized
 * Biot-Savart velocity (Eq. 1 with the cutoff of Eq. 2) and the
 * vortex-stretching term (Eq. 3), with the fast multipole method of
 * Sec. 3 (Morton octree, P2M/M2M, dual-tree traversal with the FMM MAC of
 * Algorithms 1-2, M2L, L2L/L2P, P2P) in free space or in a periodic cube
 * (Sec. 3.5).  All compute runs in CUDA kernels on the caller's stream.
 *
 * Conventions shared by every entry point
 *   - d = x_i - x_j, r = |d|, rho = r / sigma_j (the SOURCE core width),
 *     g(rho) = erf(rho/sqrt2) - sqrt(2/pi) rho exp(-rho^2/2)           (Eq. 2)
 *     u_i    = (1/4pi) sum_j g/r^3 (gamma_j x d)                         (Eq. 1)
 *     s_i    = (gamma_i . grad) u (x_i)                                  (Eq. 3)
 *   - Arrays are float32, row-major, contiguous: pos[n][3], gamma[n][3],
 *     vel[n][3], dgamma[n][3], sigma[n].  Device pointers unless the entry
 *     point name ends in _host.  The caller owns every array it passes.
 *   - Calls are asynchronous with respect to the host unless stated; they
 *     may block briefly to read small counts (tree and list sizes).
 *   - Return value: FMM_OK (0) or a negative FMM_E_* code; no call exits,
 *     traps or prints.  After an error the outputs are undefined.
 *   - A plan may be used by one host thread at a time.
 */
#ifndef FMM_VORTEX_H
#define FMM_VORTEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FMM_OK = 0,
  FMM_E_INVAL = -1,    /* bad argument (null pointer, n > n_max, p out of range ...) */
  FMM_E_NOMEM = -2,    /* device or host allocation failed */
  FMM_E_CAPACITY = -3, /* an internal list overflowed a configured bound */
  FMM_E_TIMEOUT = -4,  /* a bounded device wait gave up */
  FMM_E_DEPTH = -5,    /* translation vector outside the encodable range */
  FMM_E_CUDA = -6      /* a CUDA runtime call failed (sticky device error etc.) */
};

/* fmm_params.outputs.  FMM_OUT_STRETCHING_TRANSPOSE selects the transpose
 * scheme for dgamma: s_i = (grad u)^T gamma_i, the other reading of the
 * gradient in Eq. 3 (pair term S (gamma_i x gamma_j) + T (gamma_i . (gamma_j x d)) d;
 * with one core width it conserves the total vorticity exactly).  Without it
 * dgamma is the classical (gamma_i . grad) u. */
enum { FMM_OUT_VELOCITY = 1, FMM_OUT_STRETCHING = 2, FMM_OUT_STRETCHING_TRANSPOSE = 4 };

/* How M2L products are computed. */
enum {
  FMM_M2L_AUTO = 0,   /* tensor cores (every p) */
  FMM_M2L_SIMT = 1,   /* FP32 CUDA-core GEMM per (target tile, translation) */
  FMM_M2L_TENSOR = 2, /* tcgen05 BF16x3 split products, FP32 accumulation */
  FMM_M2L_TENSOR_TF32 = 3, /* tcgen05 TF32x3 split products (hi/lo TF32 halves, 22 bits
                              per operand), FP32 accumulation: ~16x smaller product error
                              than BF16x3 at about twice its tensor work */
  /* Flag, OR'ed with a mode: build the (tile, translation) steps by a radix
   * sort of the M2L pairs.  Without it the steps come from flag tables over
   * the translations and (tile, translation) bins whenever those tables are
   * small (compact keys of <= 22 bits, <= 2^28 bins), else from the sort.
   * Both give the same steps in the same order. */
  FMM_M2L_SORT_STEPS = 8,
  /* Flag, OR'ed with FMM_M2L_AUTO / _TENSOR: every K chunk of the BF16 M2L
   * takes the three split products.  Without it, for theta <= 0.42, source
   * degrees >= 8 take the hi x hi product only: under the MAC their terms
   * are at most theta^8 / (1 - theta) of the leading one, so that adds at
   * most 7e-6 of it (fmm_stats.m2l_split_coefs reports which). */
  FMM_M2L_FULL_SPLIT = 16,
  /* Flag: one K chunk per pipeline stage of the BF16 M2L.  Without it a step
   * of two K chunks whose second takes one product (p = 9, 10 at theta <=
   * 0.42) runs as one stage; the MMAs are the same, in the same order, so
   * the results are the same bit for bit. */
  FMM_M2L_CHUNK_STAGES = 32
};

/* fmm_params.split_tie: the cell Algorithm 1 splits when the pair's cells are
 * cubes of one size (Alg. 1 compares the two cells' radii, read here as their
 * cube sizes, and splits B unless A is the larger). */
enum {
  FMM_SPLIT_SOURCE = 0, /* split B, the source cell (Alg. 1 as printed; default) */
  FMM_SPLIT_TARGET = 1  /* split A, the target cell (an alternative, not the printed rule) */
};

/* Core width of a pair when every blob carries its own sigma (a sigma array). */
enum {
  FMM_SIGMA_SOURCE = 0, /* sigma_j of the source blob (Eq. 2 as written) */
  FMM_SIGMA_MIXED = 1   /* sigma_ij = sqrt((sigma_i^2 + sigma_j^2) / 2): symmetric in i, j */
};

typedef struct fmm_plan_s* fmm_plan;

/*
 * Parameters (Sec. 3 and 4.2).  fmm_params_default() fills the defaults.
 *   p          expansion order: degrees n = 0..p-1, p^2 real coefficients per
 *              potential; 1 <= p <= 16.  (The paper uses p = 14.)
 *   theta      MAC opening parameter: M2L iff R_A + R_B < theta |X_A - X_B|
 *              (Sec. 3.3, Fig. mac); 0 < theta < 1.
 *   ncrit      leaf capacity: a cell splits while it holds more than ncrit
 *              particles and its level is below 21 (Sec. 3.2); 1..4096.
 *   periodic   0 free space, 1 periodic cube [box_min, box_min + box_len)^3.
 *   images     periodic lattice levels: 27 explicit images through the
 *              traversal, then images-1 rings of super-cells (3^images cells
 *              per axis in total, Sec. 4.2); 1..8; ignored if !periodic.
 *   box_min, box_len   the periodic cube; ignored if !periodic.
 *   sigma_sep  k_sigma: M2L also needs |X_A-X_B| - R_A - R_B >= k_sigma *
 *              max sigma, because the far field uses the singular kernel.
 *   outputs    FMM_OUT_VELOCITY | FMM_OUT_STRETCHING, optionally
 *              | FMM_OUT_STRETCHING_TRANSPOSE (the stretching scheme); a NULL
 *              output pointer skips that output.
 *   m2l_mode   FMM_M2L_AUTO / _SIMT / _TENSOR / _TENSOR_TF32, optionally
 *              | FMM_M2L_SORT_STEPS, | FMM_M2L_FULL_SPLIT, | FMM_M2L_CHUNK_STAGES.
 *   p2p_pair_max  two leaves whose particle counts multiply to at most this
 *              do P2P even when the MAC would accept M2L (the cost rule for
 *              cells of "very few particles", Alg. 2); 0 (default): the MAC
 *              decides first; >= ncrit^2: every leaf pair does P2P (Alg. 2's
 *              printed order, leaf test before the MAC).
 *   sigma_rule FMM_SIGMA_SOURCE (default) or FMM_SIGMA_MIXED: the core width
 *              of a near-field pair when a sigma array is given (with one
 *              sigma both rules agree).  The far-field separation and the
 *              pair classes use the largest sigma, which bounds both.
 *   split_tie  FMM_SPLIT_SOURCE (default: Alg. 1's ELSE branch splits B when
 *              A and B are cubes of one size) or FMM_SPLIT_TARGET (split A
 *              then).  Alg. 1 always splits the larger cube; when that cell
 *              is a leaf the other one is split.
 *   p2p_tpl    P2P tile: target particles per lane of the one-warp pair kernel,
 *              0 (default: 2 when ncrit > 32, else 1), 1, or 2 (the two
 *              targets as the two halves of packed FP32x2 instructions).  The
 *              same pair terms either way; fmm_autotune_plan measures it.
 */
typedef struct {
  int32_t p;
  float theta;
  int32_t ncrit;
  int32_t periodic;
  int32_t images;
  double box_min[3];
  double box_len;
  float sigma_sep;
  int32_t outputs;
  int32_t m2l_mode;
  int32_t sigma_rule;
  int32_t p2p_pair_max;
  int32_t split_tie;
  int32_t p2p_tpl;
} fmm_params;

/* Work counts of the last evaluation (for throughput and roofline reports). */
typedef struct {
  int64_t n;              /* particles */
  int64_t ncells;         /* octree cells */
  int64_t nleaves;
  int32_t nlevels;        /* deepest level + 1 */
  int32_t m2l_tensor;     /* 1 if the last M2L ran on tensor cores */
  int64_t p2p_cell_pairs; /* (target leaf, source leaf, image) entries */
  int64_t p2p_pairs;      /* particle-particle interactions (incl. self pair) */
  int64_t m2l_pairs;      /* (target cell, source cell, image) M2L entries */
  int64_t m2l_steps;      /* (64-cell target tile, translation) GEMM steps */
  int64_t m2l_keys;       /* distinct translation operators */
  int64_t m2l_built;      /* operators built by this call (the rest came from the plan's cache) */
  int64_t p2p_pairs_near; /* particle pairs evaluated with the full cutoff and series test */
  int64_t p2p_pairs_mid;  /* ... with the full cutoff, rho^2 >= 2 guaranteed */
  int64_t p2p_pairs_far;  /* ... with the singular kernel, rho >= 6.5 guaranteed */
  double ms_tree;         /* phase times in ms (CUDA events), if timing enabled */
  double ms_upward;
  double ms_traverse;
  double ms_m2l;
  double ms_downward;
  double ms_p2p;
  double ms_total;
  int64_t traversal_runs; /* traversal launches (> 1 when a level outgrew the buffers) */
  int64_t m2l_split_coefs; /* tensor-core M2L: source coefficients (of P) that take all
                              three split products; the rest take hi x hi only */
  int64_t m2l_stage_chunks; /* tensor-core M2L: K chunks per pipeline stage (1, or 2
                               when a whole step runs as one stage) */
} fmm_stats;

/* Fill *prm with defaults: p=10, theta=0.4, ncrit=64, free space, images=3,
 * box [0,1)^3, sigma_sep=5, both outputs, FMM_M2L_AUTO, FMM_SIGMA_SOURCE,
 * p2p_pair_max=0, FMM_SPLIT_SOURCE. */
void fmm_params_default(fmm_params* prm);

/*
 * Create a plan for up to n_max particles on the current CUDA device.
 * Builds the M2M/L2L operators and, if periodic, the FP64 lattice operator
 * (Sec. 3.5, built on the device).  Device workspace is allocated here and grown on demand by
 * evaluations.  Returns FMM_E_INVAL for bad parameters, FMM_E_NOMEM, or
 * FMM_E_CUDA; *out is set only on success.
 */
int fmm_plan_create(const fmm_params* prm, int64_t n_max, fmm_plan* out);

/*
 * Evaluate velocity (vel) and stretching (dgamma) for n <= n_max particles.
 *   pos[n][3], gamma[n][3]   device float32 inputs (positions in the periodic
 *                             cube when periodic; free space: any finite values)
 *   sigma[n] or NULL          per-particle core widths (device); when NULL every
 *                             particle has sigma_uniform (> 0)
 *   vel[n][3], dgamma[n][3]   device float32 outputs, either may be NULL
 *   cuda_stream               cudaStream_t (NULL = legacy default stream)
 * Sec. 2.1 Eqs. (1)-(3), Sec. 3.1 (the six kernels), Algorithms 1-2.
 * Blocks the host for the small counts that size the tree and the lists.
 */
int fmm_eval_velocity_stretching(fmm_plan plan, int64_t n, const float* pos,
                                 const float* gamma, const float* sigma,
                                 float sigma_uniform, float* vel, float* dgamma,
                                 void* cuda_stream);

/*
 * Same as fmm_eval_velocity_stretching with HOST arrays: the inputs are
 * copied to plan-owned device buffers, the outputs copied back, and the call
 * returns after the stream has finished (synchronous).  Page-locked host
 * memory gives the fastest copies; pageable memory works.
 */
int fmm_eval_velocity_stretching_host(fmm_plan plan, int64_t n, const float* pos,
                                      const float* gamma, const float* sigma,
                                      float sigma_uniform, float* vel, float* dgamma,
                                      void* cuda_stream);

/*
 * Batched evaluation: nprob independent problems (no interaction between
 * them) in one pass of the method -- one forest of octrees, one traversal,
 * one set of kernel launches for all of them.  Problem k owns the particles
 * [offsets[k], offsets[k+1]) of the concatenated arrays.
 *   offsets[nprob+1]  HOST int64, offsets[0] = 0, non-decreasing,
 *                     offsets[nprob] = n <= n_max; empty problems are allowed
 *   pos, gamma        device [n][3] float32, concatenated
 *   sigma             device [n] per-particle core widths, or NULL ...
 *   sigma_prob        ... then HOST [nprob] float32, one core width per problem (> 0)
 *   boxes             HOST [nprob][4] double (box_min xyz, side) of each
 *                     periodic cube when the plan is periodic; ignored (may
 *                     be NULL) for a free-space plan, where every problem gets
 *                     its own bounding cube as in fmm_eval_velocity_stretching
 *   vel, dgamma       device [n][3] float32 outputs (either may be NULL)
 * The plan supplies p, theta, ncrit, images, sigma_sep, m2l_mode, sigma_rule
 * and p2p_pair_max for all problems.  The tree of each problem stops at level FMM_BATCH_DEPTH (16)
 * instead of 21.  The result of each problem does not depend on the other
 * problems of the batch: every sum runs in a fixed order and every constant
 * (cube, sigma, class bounds, dipole term) is the problem's own, so a problem
 * gives bit-identical outputs alone (nprob = 1) and in any batch.
 * nprob <= FMM_BATCH_MAX.  Returns FMM_E_INVAL for bad offsets, sigma or
 * boxes.  Same stream and blocking behaviour as fmm_eval_velocity_stretching.
 * (Sec. 3's method applied to many problems at once; the paper has no batch.)
 */
#define FMM_BATCH_MAX (1 << 15)
#define FMM_BATCH_DEPTH 16
int fmm_eval_batch(fmm_plan plan, int32_t nprob, const int64_t* offsets, const float* pos, const float* gamma,
                   const float* sigma, const float* sigma_prob, const double* boxes, float* vel,
                   float* dgamma, void* cuda_stream);

/*
 * Leaf-size autotuner for the batched and serving forms (the paper fixes the
 * leaf size by hand; this measures it).  For each of the ncand candidate
 * values of ncrit, a plan with base's other parameters evaluates the sample
 * batch (arguments as fmm_eval_batch, one core width per problem): one
 * untimed evaluation, then `reps` evaluations timed with CUDA events on
 * cuda_stream.  *best_ncrit receives the fastest candidate; ms_out[ncand]
 * (HOST, may be NULL) the mean milliseconds of each.  Allocates and frees
 * its own plans and output buffers; synchronous.  FMM_E_INVAL for bad
 * arguments (ncand >= 1, 1 <= reps <= 100, candidates in 1..4096).
 */
/*
 * The same measurement over leaf sizes and P2P tiles: every pair
 * (ncrit_cand[i], tpl_cand[j]) is timed as above; *best_ncrit and *best_tpl
 * receive the fastest, ms_out[n_ncrit * n_tpl] (HOST, may be NULL) the mean
 * milliseconds, ncrit-major.  tpl candidates are 0, 1 or 2 (fmm_params.p2p_tpl).
 */
int fmm_autotune_plan(const fmm_params* base, int32_t nprob, const int64_t* offsets, const float* pos,
                      const float* gamma, const float* sigma_prob, const double* boxes,
                      const int32_t* ncrit_cand, int32_t n_ncrit, const int32_t* tpl_cand, int32_t n_tpl,
                      int32_t reps, int32_t* best_ncrit, int32_t* best_tpl, double* ms_out, void* cuda_stream);
int fmm_autotune_ncrit(const fmm_params* base, int32_t nprob, const int64_t* offsets, const float* pos,
                       const float* gamma, const float* sigma_prob, const double* boxes,
                       const int32_t* candidates, int32_t ncand, int32_t reps, int32_t* best_ncrit,
                       double* ms_out, void* cuda_stream);

/* Bytes of device memory the plan holds now (its workspace grows to the
 * largest evaluation seen and is kept for the next one). */
int64_t fmm_plan_device_bytes(fmm_plan plan);

/*
 * Serving loop: a request queue in front of fmm_eval_batch (continuous
 * batching; the paper evaluates one problem per call).  Worker threads, each
 * with its own CUDA stream and device-resident plans (one per expansion order
 * and boundary type, kept between requests with their operator caches), take
 * requests as they arrive: a free worker forms a batch from the oldest queued
 * request and the later queued requests of the same (p, periodic) class, in
 * arrival order, up to max_batch_particles / max_batch_problems, and only as
 * far as the device-memory budget admits (see below).  Batches of different
 * workers run concurrently on the device.  Requests that arrive while batches
 * run wait in the queue and join the next batch of their class; a batch
 * leaves to idle workers the requests they can start at once (it takes at
 * most the queued requests minus the idle other workers).
 *
 * Memory admission: the server accounts every device byte it holds (plans and
 * staging buffers).  A batch is admitted when the bytes held by all workers,
 * with this worker's plan grown to the batch's estimated need, stay within
 * hbm_budget_bytes.  The need of a class (p, periodic) is learned from its
 * evaluations as fixed + per-particle bytes (upper envelope of what the plans
 * grew to); the first batch of a class runs alone, so its footprint is
 * measured before anything is admitted next to it.  When a batch does not fit
 * the worker first frees idle plans, then takes fewer requests, then waits
 * for other workers (which free their idle plans while anyone waits).  When
 * nothing else runs, the oldest request is attempted alone whatever its
 * estimate says; a request that does not fit the budget on its own completes
 * with FMM_E_NOMEM (see below).
 * The budget is also enforced on what the plans actually allocate: every
 * device allocation of a worker is charged to it first and refused if the
 * server's bytes would exceed hbm_budget_bytes.  A batch refused that way
 * (its class's need was underestimated) goes back to the front of the queue
 * with the class's per-particle need raised; a request refused more than 4
 * times while no other worker was running completes with FMM_E_NOMEM.  So the device bytes the server holds
 * never exceed the budget (fmm_server_counters.peak_bytes).
 *
 * batching = 0 gives the one-problem-per-call path for comparison: every
 * request is evaluated alone through fmm_eval_velocity_stretching.
 * In batching mode each result is bit-identical to the request evaluated alone
 * through fmm_eval_batch with a plan of the server's parameters.
 */
typedef struct fmm_server_s* fmm_server;

typedef struct {
  int32_t workers;              /* concurrent batches (threads + streams), 1..16 */
  int32_t batching;             /* 1 continuous batching, 0 one request per evaluation */
  int64_t hbm_budget_bytes;     /* device bytes the server may hold (> 0) */
  int64_t max_batch_particles;  /* particles per batch (a larger single request runs alone) */
  int32_t max_batch_problems;   /* requests per batch, 1..FMM_BATCH_MAX */
  float theta;                  /* as fmm_params; shared by every request */
  int32_t ncrit;                /* leaf capacity; 0: leaf capacity and P2P tile autotuned per
                                   (p, periodic) class on its first batch (fmm_autotune_plan
                                   over ncrit 32 ... 256 and p2p_tpl 1, 2) */
  float sigma_sep;
  int32_t images;
  int32_t m2l_mode;             /* the plans' other parameters take fmm_params_default's values */
  int32_t pad;
  int64_t model_bytes_per_particle; /* first estimate of a class's workspace per particle
                                       (0: 2048 bytes) until its evaluations measure it */
} fmm_server_params;

/* One request.  Host arrays; the caller keeps them valid (and does not read
 * the outputs) until fmm_server_wait reports the ticket done.  Page-locked
 * memory gives the fastest copies. */
typedef struct {
  int64_t n;             /* particles, >= 0 */
  int32_t p;             /* expansion order 1..16 */
  int32_t periodic;      /* 0 free space, 1 periodic cube `box` */
  double box[4];         /* box_min xyz, side (periodic only) */
  float sigma;           /* core width of every particle, > 0 */
  const float* pos;      /* [n][3] */
  const float* gamma;    /* [n][3] */
  float* vel;            /* [n][3] output or NULL */
  float* dgamma;         /* [n][3] output or NULL */
} fmm_request;

typedef struct {
  int32_t status;        /* FMM_OK or the FMM_E_* code of its evaluation */
  int32_t batch_problems;/* requests in the batch that carried it */
  int32_t worker;        /* worker that ran it */
  int32_t pad;
  int64_t batch_particles;
  double t_submit;       /* seconds on the server's steady clock (0 = creation) */
  double t_start;        /* batch formed */
  double t_done;         /* outputs copied back */
} fmm_request_result;

/* Server counters: batches run, requests done, particles done, the largest
 * number of device bytes the server had allocated at once, and the batches
 * that waited for memory (or were refused by the budget and re-queued). */
typedef struct {
  int64_t batches, requests, particles, peak_bytes, memory_waits;
} fmm_server_counters;

void fmm_server_params_default(fmm_server_params* prm); /* 2 workers, batching, 64 GiB, 16M particles,
                                                           4096 problems, theta 0.5, ncrit 64,
                                                           sigma_sep 5, images 3, AUTO */
int fmm_server_create(const fmm_server_params* prm, fmm_server* out);  /* current CUDA device */
/* Queue a request; *ticket identifies it.  FMM_E_INVAL for a bad request. */
int fmm_server_submit(fmm_server srv, const fmm_request* req, int64_t* ticket);
/* Wait up to timeout_s seconds (< 0: no limit) for a ticket; FMM_OK and *out
 * filled once done (the ticket is then forgotten), FMM_E_TIMEOUT if not done
 * yet, FMM_E_INVAL for an unknown ticket.  The request's own status is out->status. */
int fmm_server_wait(fmm_server srv, int64_t ticket, double timeout_s, fmm_request_result* out);
/* Seconds on the server's clock (for arrival schedules). */
double fmm_server_clock(fmm_server srv);
int fmm_server_get_counters(fmm_server srv, fmm_server_counters* out);
/* Finish queued work, stop the workers, free everything.  NULL is ok. */
void fmm_server_destroy(fmm_server srv);

/* Release every resource of the plan (synchronizes the device). NULL is ok. */
void fmm_plan_destroy(fmm_plan plan);

/* Static string for an FMM_* code. */
const char* fmm_strerror(int code);

/*
 * Velocity at nt target points from ns source blobs (Sec. 4.3 compares the
 * kinetic energy spectrum of the vortex-method field with the spectral
 * method's, which needs the velocity on grid points that are not particles).
 *   src_pos[ns][3], src_gamma[ns][3]   device float32 sources
 *   src_sigma[ns] or NULL              per-source core widths, or sigma_uniform (> 0)
 *   tgt_pos[nt][3]                     device float32 target points (inside the
 *                                      periodic cube when the plan is periodic)
 *   vel[nt][3]                         device float32 output
 * The targets join the plan's tree as blobs of zero strength behind the
 * sources (ns + nt <= n_max), so the result is the field of the sources alone
 * evaluated by the same FMM; a target that coincides with a source gets the
 * regularized field there.  Velocity only.  Per-source core widths: the
 * targets take the largest source width, so the far-field separation and
 * the pair classes are those of the sources; pairs take the source width
 * sigma_j whatever the plan's sigma_rule (a point has no width of its own).  Same stream and blocking
 * behaviour as fmm_eval_velocity_stretching; FMM_E_INVAL for bad arguments.
 */
int fmm_eval_targets(fmm_plan plan, int64_t ns, const float* src_pos, const float* src_gamma,
                     const float* src_sigma, float sigma_uniform, int64_t nt, const float* tgt_pos,
                     float* vel, void* cuda_stream);

/*
 * Re-evaluation with new strengths on the plan's last tree.  The vortex
 * method re-initialises its particles onto the same positions every step, so
 * the tree structure is built once and reused (Sec. 3.4).  After a full
 * evaluation (fmm_eval_velocity_stretching or fmm_eval_batch) of n particles,
 * this call evaluates velocity and stretching for the SAME positions and core
 * widths and new strengths:
 *   gamma[n][3]            device float32, in the caller's particle order
 *   vel[n][3], dgamma[n][3] device float32 outputs (either may be NULL)
 * It keeps the sorted positions, octree, interaction lists and M2L operators
 * of that evaluation and runs only the strength-dependent steps (gather of
 * the strengths into the sorted order, P2M/M2M, M2L, periodic lattice
 * operator and dipole term, L2L/L2P, P2P and the combine), with the same
 * kernels in the same order, so the result is bit-identical to a full
 * evaluation of the same input.  Fully asynchronous on cuda_stream: no host
 * synchronization, no allocation; errors raised by kernels (FMM_E_TIMEOUT)
 * are kept on the device and read by fmm_plan_status.  FMM_E_INVAL if the
 * plan's last call was not a successful full evaluation (or was
 * fmm_eval_targets, whose tree also holds the targets).
 */
int fmm_eval_strengths(fmm_plan plan, const float* gamma, float* vel, float* dgamma,
                       void* cuda_stream);

/*
 * The error status raised on the device by the plan's last evaluation
 * (FMM_OK or FMM_E_TIMEOUT): waits for cuda_stream, then reads one int.
 */
int fmm_plan_status(fmm_plan plan, void* cuda_stream);

/*
 * A CUDA graph of fmm_eval_strengths for fixed buffers: the call's kernel
 * launches are recorded once (stream capture) and replayed by
 * fmm_graph_launch, one graph launch per evaluation, nothing on the host in
 * between.  gamma, vel and dgamma are the device arrays every replay reads
 * and writes: write the next strengths into gamma (stream-ordered), launch,
 * read vel/dgamma.  The graph is tied to the plan's current tree: a later
 * full evaluation on the plan makes fmm_graph_launch return FMM_E_INVAL
 * (capture again).  Destroy graphs before their plan.
 */
typedef struct fmm_graph_s* fmm_graph;
int fmm_graph_capture(fmm_plan plan, const float* gamma, float* vel, float* dgamma, fmm_graph* out);
int fmm_graph_launch(fmm_graph graph, void* cuda_stream);
/* Kernel launches one replay performs (counted in fmm_kernel_launch_count). */
int64_t fmm_graph_kernel_count(fmm_graph graph);
void fmm_graph_destroy(fmm_graph graph);

/*
 * The periodic lattice operator of a plan (Sec. 3.5): the P x P (P = p^2) FP64
 * matrix A, row-major, with L~_root += A M~_root in the normalized
 * real-packed coefficients: the images beyond the 27 explicit ones, as
 * images-1 rings of 702 super-cells (sides 1, 3, 9 ... in box units).  Plans
 * build it on the device in FP64 (on_device = 1, what plans use); on_device
 * = 0 builds the same sums on the host in FP64, for comparison.  out: host
 * [p^4] doubles.  Synchronous; FMM_E_INVAL for p outside 1..16 or images
 * outside 1..8.
 */
int fmm_lattice_operator(int32_t p, int32_t images, int32_t on_device, double* out);

/*
 * Measurement aid (no counterpart in the paper): the FP32 rate the device
 * sustains on independent packed FMA chains (FFMA2), in TFLOP/s (FMA = 2
 * flops), timed with CUDA events over `launches` launches (1..1000) of a
 * kernel with 8 CTAs of 256 threads per SM.  Synchronous.  It is the
 * practical ceiling beside the derived peak (FP32 lanes x clock) that the
 * P2P roofline fraction is quoted against.
 */
int fmm_probe_fp32_rate(int32_t launches, double* tflops, double* ms_per_launch, void* cuda_stream);

/*
 * All-pairs direct sum of Eqs. (1)-(3) on the device, free space, without
 * a tree: the same P2P pair kernel over every (target, source) pair of one
 * array (the self pair excluded).  Device arrays as above.  O(n^2).
 */
int fmm_direct_velocity_stretching(int64_t n, const float* pos, const float* gamma,
                                   const float* sigma, float sigma_uniform, float* vel,
                                   float* dgamma, void* cuda_stream);

/*
 * Allocation-free Morton ordering, for callers that cannot call cudaMalloc:
 * code under a memory manager that owns every device allocation (a framework
 * caching allocator, a fixed device-memory budget) or code that must not
 * trigger the implicit device-wide synchronization cudaMalloc / cudaFree can
 * cause.  The paper has no counterpart of this entry point.
 *
 * Computes the cube (free space: as the plans do; periodic: the given cube),
 * the 63-bit Morton key of every position (21 bits per axis, x most
 * significant) and a stable sort of (key, index):
 *   pos[n][3]     device float32 positions (input)
 *   periodic      0: free-space cube from the bounding box; 1: box_min/box_len
 *   box_min[3]    HOST array, read only when periodic
 *   keys_out[n]   device, the sorted keys
 *   order_out[n]  device, sorted position -> input index
 * Identical results to the ordering fmm_eval_velocity_stretching computes
 * (see fmm_plan_get_order).  Allocates nothing: every temporary lives in one
 * static device array of about 12.4 MB that exists on every GPU that loads
 * the library until the process exits.  n must be <= FMM_NOALLOC_MAX_N;
 * larger n returns FMM_E_CAPACITY and launches nothing.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress, with the device current); make that
 * first call before any stream capture.  Host threads may make that first
 * call at the same time (the cached address is atomic).  All calls share the array and it
 * keeps the last call's contents; calls whose GPU work overlaps (other
 * streams, other threads) race on it and give undefined results.  Nothing in
 * the array needs to start at zero.  Asynchronous on cuda_stream.
 */
#define FMM_NOALLOC_MAX_N (1 << 20)
int fmm_morton_order_noalloc(int64_t n, const float* pos, int periodic, const double* box_min,
                             double box_len, uint64_t* keys_out, uint32_t* order_out,
                             void* cuda_stream);

/*
 * Self-test of the bounded device wait that guards every mbarrier wait of the
 * tensor-core M2L kernel (a wait that gives up records FMM_E_TIMEOUT instead of
 * hanging, and the kernel returns).  One thread of one CTA waits on a shared
 * memory barrier with at most `spins` polls (1 .. 2^24): arrive = 1 completes
 * the barrier first (returns FMM_OK), arrive = 0 leaves it incomplete so the
 * wait runs out (returns FMM_E_TIMEOUT).  Synchronous; FMM_E_INVAL for bad
 * arguments.  The CUDA context stays usable afterwards.
 */
int fmm_selftest_bounded_wait(int64_t spins, int arrive, void* cuda_stream);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all plans and entry points; for launch accounting in benchmarks). */
int64_t fmm_kernel_launch_count(void);

/*
 * Starting capacities (entries) of the traversal's buffers for the plan's
 * next evaluations: the frontier, the M2L pairs and the P2P pairs (0: sized
 * from the cell count and what the plan's earlier evaluations needed, the
 * default).  The traversal runs all levels in one launch; when a level's
 * output would outgrow a buffer the launch stops before writing it, the
 * buffers grow (contents kept) and a new launch resumes at that level
 * (fmm_stats.traversal_runs counts the launches).  Small values exercise
 * that path.  FMM_E_INVAL for a negative value.
 */
int fmm_plan_set_list_capacity(fmm_plan plan, int64_t frontier, int64_t m2l, int64_t p2p);

/* Enable (1) or disable (0) CUDA-event phase timing in fmm_stats. */
int fmm_plan_set_timing(fmm_plan plan, int enable);

/* Work counts and phase times of the last evaluation (synchronizes). */
int fmm_plan_get_stats(fmm_plan plan, fmm_stats* out);

/*
 * Inspection of the last evaluation's tree and lists (synchronizes, copies
 * to HOST arrays the caller sized from fmm_plan_get_stats).  Any pointer may
 * be NULL to skip it.
 *   order[n]  sorted position -> input index;  keys[n]  sorted Morton keys
 *   per cell: begin, end (sorted particle range), level, parent, child_begin,
 *   nchild, center[3] (FP64 cube centre), radius (FP64)
 *   p2p[m][3] / m2l[m][3]: (target cell, source cell, image 0..26; 13 = none)
 *   in traversal order (P2P grouped by target leaf).
 */
int fmm_plan_get_order(fmm_plan plan, uint32_t* order, uint64_t* keys);
int fmm_plan_get_cells(fmm_plan plan, int32_t* begin, int32_t* end, int32_t* level,
                       int32_t* parent, int32_t* child_begin, int32_t* nchild,
                       double* center, double* radius);
int fmm_plan_get_lists(fmm_plan plan, int32_t* p2p, int32_t* m2l);

#ifdef __cplusplus
}
#endif

#endif /* FMM_VORTEX_H */
