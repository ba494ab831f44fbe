/*
 * jkcals.h -- C ABI of the GB300-native JK-CALS library (libjkcals.so).
 *
 * JK-CALS (Psarras, Karlsson, Bro, Bientinesi, "Accelerating jackknife
 * resampling for the Canonical Polyadic Decomposition") fits every jackknife
 * submodel of a CP model at once.  Each submodel g leaves out a set D_g of
 * samples (indices of the sampled mode n_hat; leave-one-out: D_g = {g}).  Its
 * factor matrices sit side by side in "multi-matrices" Ubar^(n) (I_n x C,
 * C = sum_g R_g), and rows D_g of block g of Ubar^(n_hat) are kept at zero, so
 * that one MTTKRP with the *full* tensor serves every resampled tensor
 * (Sec. 4.1, Case I and Case II; Alg. 3).
 *
 * Notation used below: N modes (order of the tensor), dims I_0..I_{N-1}
 * (0-based: mode n here is mode n+1 of the paper), K blocks (submodels),
 * R_g components of block g, C = sum_g R_g, block g owns columns
 * [off_g, off_g + R_g) with off_g = R_0 + ... + R_{g-1}.
 *
 * Conventions shared by every call:
 *  - Memory.  Every pointer argument that carries data (tensor, factors,
 *    outputs) may point to host memory or to device memory of the handle's
 *    device; the library copies with unified addressing (cudaMemcpyDefault).
 *    The caller owns those buffers.  The library owns its workspace, its own
 *    copies of the tensor and factors, and its CUDA graphs.
 *  - Layouts.  The tensor is dense C-order (last index fastest), FP64 or FP32.
 *    Factor multi-matrices are row-major I_n x C, FP64.
 *  - Streams.  Work is enqueued on the stream given at create (NULL = the
 *    legacy default stream).  Calls that return values in host memory
 *    synchronise that stream before returning.
 *  - Errors.  Every call returns a jkcals_status and never throws across the
 *    ABI.  jkcals_last_error() gives a thread-local message for the last
 *    failing call of the calling thread.  A sticky CUDA error maps to
 *    JKCALS_ERR_CUDA and leaves the handle in the STATE error (destroy only).
 *  - Threads.  A handle may be used by one thread at a time.
 */
#ifndef JKCALS_H
#define JKCALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jkcals_ctx* jkcals_t;

typedef enum {
  JKCALS_OK = 0,
  JKCALS_ERR_ARG = 1,         /* invalid argument; nothing was enqueued          */
  JKCALS_ERR_CUDA = 2,        /* a CUDA runtime/driver call failed               */
  JKCALS_ERR_OOM = 3,         /* device allocation failed (or hit the cap)       */
  JKCALS_ERR_NOT_SPD = 4,     /* some submodel met a non-SPD H (see block status) */
  JKCALS_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                   */
  JKCALS_ERR_STATE = 6,       /* handle unusable after an earlier fatal error    */
  JKCALS_ERR_UNSUPPORTED = 7  /* valid but outside this build's limits           */
} jkcals_status;

/* Arithmetic of the concurrent MTTKRP (Alg. 3 MTTKRP line).  The Gram,
 * Cholesky, solve, normalisation and error kernels are FP64 in every form.  */
typedef enum {
  JKCALS_FP64 = 0,        /* FP64 products and sums (CUDA cores)                       */
  JKCALS_TF32 = 1,        /* tcgen05 kind::tf32, FP32 accumulation in TMEM             */
  JKCALS_3XTF32 = 2,      /* hi*hi + hi*lo + lo*hi TF32 products, FP32 accumulation    */
  JKCALS_BF16 = 3,        /* tcgen05 kind::f16 with BF16 operands, FP32 accumulation   */
  JKCALS_SPLIT_BF16 = 4,  /* BF16 hi/mid/lo split, 6 cross products, FP32 accumulation */
  JKCALS_EXACT_BF16 = 5   /* exact-chain sliced BF16: every operand row is cut into four
                             7-bit integer slices on a shared power-of-two grid, stored as
                             BF16; the two leading product levels accumulate exactly in
                             FP32 TMEM (chains <= 1024 terms), the smaller levels beside
                             them; chains are combined as FP32 pairs (double-float) and
                             the split-K partials summed into FP64.  Modes of <= 128 rows
                             whose largest other mode has >= 128 run a two-step variant
                             (GEMMs against the sliced rows of that mode, scaled by the
                             remaining modes' entries).  Measured accuracy: MTTKRP
                             within ~2e-9 relative of FP64 (tested at 1e-8 element by
                             element), factors within ~4e-8 of the FP64 path after 100
                             sweeps of the 300x100x50 workload (tested at 1e-6); not the
                             FP64 form's 1e-12.  10 BF16 MMA passes per product. */
} jkcals_prec;

typedef enum { JKCALS_DTYPE_F32 = 0, JKCALS_DTYPE_F64 = 1 } jkcals_dtype;

/* Per-block status bits (jkcals_get_block_status). */
#define JKCALS_BLOCK_NOT_SPD 1    /* Cholesky failed; block frozen since          */
#define JKCALS_BLOCK_CONVERGED 2  /* tolerance test met; block frozen since       */

typedef struct {
  int precision;        /* jkcals_prec, default JKCALS_FP64                               */
  int normalise;        /* 1 (default): after updating mode n < N-1, scale each column of
                           every block to unit 2-norm (a zero column is left as is)       */
  int use_graph;        /* 1 (default): replay sweeps from a captured CUDA graph          */
  int splits;           /* 0 (default) = automatic split-K factor of the MTTKRP, else fixed */
  int64_t max_device_bytes; /* 0 (default) = no cap; > 0: allocations beyond this many bytes
                               fail with JKCALS_ERR_OOM (lets callers bound device memory) */
  int kernel_timing;    /* 1: record CUDA events around every MTTKRP launch of a sweep
                           (read with jkcals_kernel_times); 0 (default): off            */
  int update_mode;      /* per-block update kernels: 0 (default) automatic, 1 one CTA per
                           block with the block's rows in shared memory, 2 two-phase
                           (row chunks, then a per-block reduction)                    */
  int autotune;         /* 1: at create, time the MTTKRP (+ split-K reduction) of every mode
                           for split factors around the planned one and keep the fastest
                           (ignored when splits > 0); 0 (default): off                   */
  int compact;          /* 1 (default): inside jkcals_run, once at most half of the blocks
                           being swept are still active, lay the active blocks out side by
                           side and sweep only them (the MTTKRP then spans only their
                           columns); the full layout is restored before jkcals_run returns.
                           0: converged blocks keep their columns until the end           */
  int batch_branches;   /* 0 (default): a batch (jkcals_batch_create) whose handles share one
                           tensor-core form and order runs each kernel step of all problems
                           as one grouped launch; 1 on any handle of a batch: the batch runs
                           every problem's own sweep graph as a parallel branch instead     */
  int reserved[3];
} jkcals_options;

/* Fill *opt with the defaults above. */
void jkcals_default_options(jkcals_options* opt);

/*
 * jkcals_create -- Alg. 3 initialisation (the loop that builds one factor
 * multi-matrix per mode): copy the tensor into per-mode unfoldings T_(n)
 * (Sec. 3.1, columns ordered by Eq. kolda_mapping), compute ||T_{-g}||^2 for
 * the error line of Alg. 3, copy the initial multi-matrices, zero rows D_g of
 * block g in mode sampled_mode (Alg. 3, red branch of the initialisation) and
 * compute the per-block Grams.
 *
 *  out           receives the handle (NULL on failure)
 *  N, dims       order (1 <= N <= 8 ... see limits) and the N dims, each >= 1
 *  T, T_dtype    dense C-order tensor, host or device, JKCALS_DTYPE_F32/F64;
 *                copied during the call, may be freed on return
 *  sampled_mode  n_hat, 0 <= sampled_mode < N
 *  K, ranks      number of blocks (>= 1) and R_g for each (1 <= R_g <= 32)
 *  left_out_ptr  K+1 offsets into left_out_idx (CSR, left_out_ptr[0] = 0)
 *  left_out_idx  the indices D_g, each in [0, dims[sampled_mode]); an empty
 *                set makes block g the model of the full tensor
 *  init          N pointers, init[n] is the I_n x C row-major FP64 initial
 *                multi-matrix (host or device), copied during the call
 *  opt           options or NULL for the defaults
 *  stream        cudaStream_t as void*, NULL = legacy default stream
 *
 * Device memory comes from the library's stream-ordered memory pool of the
 * current device (allocated on the handle's stream; the call returns after
 * the stream is idle).  Memory freed by destroyed handles stays in that pool,
 * up to 2 GiB per device, for the next handle; more is returned to the device
 * at synchronisation points.  Without pool support the handle uses cudaMalloc.
 *
 * Limits: N <= 8, R_g <= 32, prod(dims) < 2^40.
 * Errors: ARG on any invalid value, OOM, CUDA, UNSUPPORTED (limits).
 */
jkcals_status jkcals_create(jkcals_t* out, int N, const int64_t* dims, const void* T, int T_dtype,
                            int sampled_mode, int K, const int32_t* ranks,
                            const int64_t* left_out_ptr, const int64_t* left_out_idx,
                            const double* const* init, const jkcals_options* opt, void* stream);

/* Release every resource of the handle (NULL is ignored): its device memory
 * goes back to the library's pool in the order of the handle's stream.
 * Synchronises the stream.  A batch that holds the handle must be destroyed
 * first. */
void jkcals_destroy(jkcals_t h);

/*
 * jkcals_mttkrp -- the concurrent MTTKRP of Alg. 3 (MTTKRP line):
 *   Mbar_n = T_(n) (Ubar^(N-1) (.) ... (.) Ubar^(n+1) (.) Ubar^(n-1) (.) ... (.) Ubar^(0))
 * for the handle's current multi-matrices, in the handle's precision.  Block
 * g's columns equal submodel g's own MTTKRP on its sliced tensor (Sec. 4.1);
 * for mode == sampled_mode rows D_g of block g are the full-tensor values that
 * Case I discards.
 *  M_out   I_mode x C row-major FP64, host or device.
 * Errors: ARG (mode out of range, NULL), CUDA, STATE.
 */
jkcals_status jkcals_mttkrp(jkcals_t h, int mode, double* M_out);

/*
 * jkcals_als_sweep -- nsweeps iterations of the repeat loop of Alg. 3: for
 * every mode n, the concurrent MTTKRP, then per block the Hadamard of Grams,
 * the Cholesky solve of the update line, zeroing of rows D_g in the sampled
 * mode, column normalisation (modes n < N-1, if enabled) and the Gram
 * refresh; after the last mode, the per-block error of the Alg. 3 error line
 * (read with '+' before the model-norm term):
 *   e_g = ||T_{-g}||^2 + sum(H_{N-1,g} * G_{N-1,g}) - 2 sum(Ubar_{N-1|g} * Mbar_{N-1|g}).
 * Blocks frozen (NOT_SPD or CONVERGED) keep their factors; their losses are NaN.
 *  losses  NULL or nsweeps x K FP64 (host or device): e_g after each sweep.
 * Returns NOT_SPD if any block has the NOT_SPD bit after the call (the other
 * blocks were still advanced); OK otherwise.
 */
jkcals_status jkcals_als_sweep(jkcals_t h, int nsweeps, double* losses);

/*
 * jkcals_als_sweep_async -- the sweeps of jkcals_als_sweep, only enqueued on the
 * handle's stream: no host synchronisation and no status check (read the block
 * status with jkcals_get_block_status).
 *  losses_dev  NULL or nsweeps x K FP64 in device memory.
 */
jkcals_status jkcals_als_sweep_async(jkcals_t h, int nsweeps, double* losses_dev);

/*
 * jkcals_kernel_times -- device time of each mode's concurrent MTTKRP launch in
 * the last completed sweep (requires opt.kernel_timing = 1; synchronises).
 *  ms  N doubles (host), milliseconds per mode.
 */
jkcals_status jkcals_kernel_times(jkcals_t h, double* ms);

/*
 * jkcals_sweep_info -- how one sweep is executed on the device.
 *  kernels_per_sweep  receives the number of kernel launches of one sweep
 *  splits             NULL or N ints (host): the split-K factor of each mode's MTTKRP
 */
jkcals_status jkcals_sweep_info(jkcals_t h, int* kernels_per_sweep, int* splits);

/*
 * jkcals_jackknife_se -- Alg. 2 post-processing on the device: every jackknife
 * submodel (block with a non-empty left-out set, G of them, in block order) is
 * adjusted to a reference model (Alg. 2 adjustment line: in every mode but the
 * last, the entry of largest magnitude of each column made positive, the flip
 * carried into the last mode; then the column permutation maximising
 * sum_s prod_{n != sampled_mode} |cos(submodel column perm[s], reference column s)|,
 * over all R! permutations for R <= 8 with ties to the lexicographically first,
 * by the Hungarian method for R > 8), and the jackknife standard error
 * S_n = sqrt((G-1)/G sum_g (U_n^g - mean_g U_n^g)^2) of every entry is formed
 * (Alg. 2 std line) for the modes n != sampled_mode.  Uses the handle's current
 * factors; synchronises.
 *  ref_block    >= 0: the reference is that block's current factors (e.g. the full model
 *               fitted in the same handle); < 0: ref gives it
 *  ref          N pointers (host or device), row-major I_n x R FP64; ignored when ref_block >= 0
 *  S            N pointers (host or device), row-major I_n x R FP64; S[sampled_mode] may be
 *               NULL and is not written
 *  perm         NULL or G x R int32 (host or device): reference column s <- submodel column perm[g][s]
 *  aligned      NULL or N pointers (host or device), G x I_n x R FP64 (submodel-major):
 *               the adjusted submodels
 *  n_submodels  NULL or receives G
 * Errors: JKCALS_ERR_ARG when fewer than two submodels, when the submodels (and the
 * reference block) differ in rank, or for NULL arguments; JKCALS_ERR_OOM for the
 * workspace (G + 2) x sum_n I_n x R doubles.
 */
jkcals_status jkcals_jackknife_se(jkcals_t h, int ref_block, const double* const* ref, double* const* S,
                                  int32_t* perm, double* const* aligned, int* n_submodels);

/*
 * jkcals_mode_plan -- how one mode's concurrent MTTKRP (Alg. 3 MTTKRP line) runs.
 *  mode          0 <= mode < N, else JKCALS_ERR_ARG
 *  kernel        receives 0 (FP64 on the CUDA cores), 1 (tensor cores, the Khatri-Rao
 *                tile built in shared memory), 2 (exact-chain two-step form: one GEMM
 *                against the sliced rows of mode fastest_mode per index of the remaining
 *                modes, scaled by their factor entries in the epilogue)
 *  tile_rows     NULL or receives the rows of the mode per CTA (N tile)
 *  stages        NULL or receives the operand pipeline depth (0 for FP64)
 *  fastest_mode  NULL or receives the other mode that runs fastest along the columns
 *                of the operand layout (-1 for FP64)
 */
jkcals_status jkcals_mode_plan(jkcals_t h, int mode, int* kernel, int* tile_rows, int* stages,
                               int* fastest_mode);

/*
 * jkcals_plan_query -- the plan jkcals_create would make, computed on the host alone
 * (no device, no allocation, no handle): a tensor of N modes of sizes dims, K blocks of
 * the given ranks, the options' precision and split setting, on a GPU of num_sms SMs.
 *  kernel     N ints (host): per mode 0 (FP64), 1 (tensor cores, one-step), 2 (two-step)
 *  tile_rows  NULL or N ints: rows of the mode per CTA
 *  stages     NULL or N ints: operand pipeline depth (0 for FP64)
 *  splits     NULL or N ints: split-K factor of the MTTKRP
 * Errors: JKCALS_ERR_ARG for bad sizes or options; JKCALS_ERR_UNSUPPORTED where
 * jkcals_create would refuse the shape (rank > 32, tiles or grids beyond the limits).
 */
jkcals_status jkcals_plan_query(int N, const int64_t* dims, int K, const int32_t* ranks,
                                const jkcals_options* opt, int num_sms, int* kernel, int* tile_rows,
                                int* stages, int* splits);

/*
 * jkcals_run -- sweeps until every block is frozen or max_sweeps is reached.
 * With tol > 0 a block converges when |e_prev - e| / ||T_{-g}||^2 < tol
 * (stopping rule of Alg. 1/Alg. 3) and is frozen from then on.
 *  sweeps_done  NULL or receives the number of sweeps run (host)
 *  final_loss   NULL or K FP64 (host or device): the last finite e_g per block
 */
jkcals_status jkcals_run(jkcals_t h, int max_sweeps, double tol, int* sweeps_done,
                         double* final_loss);

/*
 * Sweeps each block ran in the latest jkcals_run (K int32, host): a block that
 * converged (or met a non-positive pivot) stops counting at the sweep that
 * froze it -- with tol > 0 the sweep count at which the stopping rule of Alg. 1
 * (Sec. 3.2) held for it.  JKCALS_ERR_STATE before the first jkcals_run.
 */
jkcals_status jkcals_run_block_sweeps(jkcals_t h, int32_t* sweeps);

/* Copy the current multi-matrices out: U[n] is I_n x C row-major FP64 (host or device). */
jkcals_status jkcals_get_factors(jkcals_t h, double* const* U);

/* Replace the multi-matrices (checkpoint resume); rows D_g of the sampled mode are
 * zeroed again and the Grams recomputed.  Clears the CONVERGED bits and the stored
 * previous losses.  U[n]: I_n x C row-major FP64 (host or device). */
jkcals_status jkcals_set_factors(jkcals_t h, const double* const* U);

/* Per-block status bits (JKCALS_BLOCK_*), K int32 (host). */
jkcals_status jkcals_get_block_status(jkcals_t h, int32_t* status);

/*
 * jkcals_grad -- gradient of the summed reconstruction loss over all blocks,
 *   f = sum_g ||T_{-g} - [[Ubar^(0)_{|g}, ..., Ubar^(N-1)_{|g}]]||^2,
 * at the multi-matrices U (NULL = the handle's current ones; U is then taken
 * with rows D_g of the sampled mode zeroed).  The gradient of block g with
 * respect to Ubar^(n)_{|g} is 2 (Ubar^(n)_{|g} H^(n)_g - Mbar_{n|g}) (the
 * normal equations of the update line of Alg. 1 written as a gradient), with
 * Mbar_n the concurrent MTTKRP; rows D_g of the sampled mode get 0.
 *  G     N pointers, G[n] is I_n x C row-major FP64 (host or device), or NULL
 *  loss  NULL or one FP64 in host memory: f
 */
jkcals_status jkcals_grad(jkcals_t h, const double* const* U, double* const* G, double* loss);

/*
 * Batched problems (many independent jackknife problems, each its own handle;
 * configuration 4 of the evaluation).  The paper fits one tensor at a time;
 * batching is a deployment form of Alg. 3 for many small problems, none of
 * which fills the GPU alone.  A sweep of the whole batch is one CUDA graph
 * launch.  When every handle uses the same tensor-core form, the same tensor
 * order and the one-step MTTKRP in every mode (and none sets
 * opt.batch_branches), the graph holds grouped launches: per mode, one MTTKRP
 * launch over the tiles of all problems (a CTA finds its problem and tile in a
 * prefix table of tile counts), one fused-update launch per class of
 * (largest rank, uniform ranks), the remaining problems' reduction and
 * two-phase update, then one launch that advances every sweep counter.  If any
 * handle set opt.autotune, the split-K factor of every problem is scaled by 1,
 * 1/2, 1/4 or 1/8 per mode, each grouped MTTKRP timed, and the fastest kept.
 * Otherwise each handle's own sweep is captured and the captures become
 * parallel branches (child graphs) of the batch's graph.  Both forms compute
 * each problem's sweep exactly as jkcals_als_sweep does (same plans, same
 * summation order).
 *  handles     n handles, owned by the caller, alive for the batch's lifetime;
 *              no handle may have opt.kernel_timing = 1
 *  max_sweeps  the most sweeps one jkcals_batch_sweep call may run (each
 *              handle's loss history is sized for it now)
 *  stream      cudaStream_t the batch runs on (NULL: the batch creates its own)
 * jkcals_batch_sweep enqueues nsweeps sweeps of every problem, ordered after
 * the work already enqueued on each handle's stream and before later work
 * there; it does not synchronise.  Read each problem's losses with
 * jkcals_loss_history and its factors with jkcals_get_factors.  A handle whose
 * loss history was reallocated since (a jkcals_als_sweep call for more sweeps
 * than max_sweeps) makes jkcals_batch_sweep return JKCALS_ERR_STATE.
 */
typedef struct jkcals_batch_ctx* jkcals_batch_t;
jkcals_status jkcals_batch_create(jkcals_batch_t* out, int n, const jkcals_t* handles, int max_sweeps,
                                  void* stream);
jkcals_status jkcals_batch_sweep(jkcals_batch_t b, int nsweeps);
jkcals_status jkcals_batch_sync(jkcals_batch_t b);
void jkcals_batch_destroy(jkcals_batch_t b);

/*
 * Losses e_g of the last nsweeps sweeps run by the latest jkcals_als_sweep,
 * jkcals_als_sweep_async or jkcals_batch_sweep call (nsweeps x K, sweep-major;
 * host or device; synchronises when losses is host memory).
 */
jkcals_status jkcals_loss_history(jkcals_t h, int nsweeps, double* losses);

/*
 * Self-test of the bounded waits that every pipelined kernel relies on (a
 * health check; no counterpart in the paper).  One CTA on the current device:
 * one thread waits on a barrier phase that nothing completes, with a limit of
 * limit_ms (0 < limit_ms <= 100); it must give up, raise the CTA's abort flag
 * and record its code (3) in the error word.  A thread of another warp,
 * blocked in a wait with a limit 64 times longer, must leave through the abort
 * flag.  No trap and no fault: the kernel returns and the context stays
 * usable.
 *  code           the error word the kernel recorded (3 when the wait expired as designed)
 *  left_after_ms  time from the start until the second thread left its wait (about limit_ms)
 * Returns JKCALS_OK after the kernel completed and neither wait claimed a
 * completion that never happened; JKCALS_ERR_STATE if one did; JKCALS_ERR_ARG
 * or JKCALS_ERR_CUDA otherwise.  Synchronises the device.
 */
jkcals_status jkcals_selftest_bounded_wait(double limit_ms, int* code, double* left_after_ms);

/* Block until the handle's stream is idle. */
jkcals_status jkcals_sync(jkcals_t h);

/*
 * jkcals_mttkrp_f64_noalloc -- the FP64 concurrent MTTKRP of one mode for callers
 * that cannot allocate device memory.  The paper has no counterpart: it is a
 * deployment variant of the same computation as jkcals_mttkrp.  Callers such as
 * a solver that runs inside someone else's memory pool or arena, a step whose
 * memory budget was fixed in advance, or a latency-critical loop in which a
 * cudaMalloc would synchronise the device cannot create a handle, because a
 * handle allocates its own tensor copies and workspace.  This entry point
 * allocates nothing: the caller passes every input and the output, and the
 * split-K partial sums go to a fixed scratch array that the library keeps in
 * device memory.
 *
 *   M_out = Tn (U[N-1] (.) ... (.) U[mode+1] (.) U[mode-1] (.) ... (.) U[0])
 *
 *  N, dims  order (2..8) and the N dims (host)
 *  mode     the mode whose MTTKRP is computed
 *  Tn       device, I_mode x J row-major FP64 with J = prod_{k != mode} dims[k]:
 *           the mode-`mode` unfolding, column j holding the element whose other
 *           indices satisfy j = sum_{k != mode} i_k prod_{m < k, m != mode} dims[m]
 *  U        N pointers (host array) to device I_k x C row-major FP64 matrices;
 *           U[mode] is not read and may be NULL
 *  C        columns of every U[k] and of M_out
 *  M_out    device, I_mode x C row-major FP64, overwritten
 *  stream   cudaStream_t as void*, NULL = legacy default stream
 *
 * Scratch: a file-scope device array of 2^21 doubles (16 MiB), which every GPU
 * that loads the library holds until the process exits.  Calls with
 * dims[mode] * C > 2^21 return JKCALS_ERR_UNSUPPORTED.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, no
 * allocation); make that first call before any stream capture.  Every call
 * shares the array and overwrites, before reading, every element it uses, so
 * the previous call's leftovers never matter; but calls whose work overlaps on
 * the GPU (other streams, other host threads) race on the array and give wrong
 * results: serialise them, e.g. on one stream.  The looked-up address is kept
 * for the life of the process: after cudaDeviceReset (or any teardown of the
 * device's primary context) the entry point must not be called again in that
 * process.  Tn, U[k] and M_out must be device (or managed) memory of the
 * current device; host pointers and pointers into another GPU's memory are
 * rejected with JKCALS_ERR_ARG.  Returns after enqueueing (no sync).
 */
jkcals_status jkcals_mttkrp_f64_noalloc(int N, const int64_t* dims, int mode, const double* Tn,
                                        const double* const* U, int C, double* M_out, void* stream);

/* Thread-local message of the last failing call ("" if none). */
const char* jkcals_last_error(void);

/* Library version string. */
const char* jkcals_version(void);

#ifdef __cplusplus
}
#endif
#endif /* JKCALS_H */
