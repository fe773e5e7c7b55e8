/*
 * ttprice -- tensor-train Fourier pricer for multi-asset European options
 * (arXiv 2203.02804), GB300 / sm_103a.
 *
 * What it computes.  For d correlated GBM assets (Section II.A: dS^j = r S^j dt
 * + sigma_j S^j dW^j with annualised covariance Cov) the price of a call on the
 * minimum (Eq. minpayoff) is the damped d-dimensional Fourier integral of
 * Eq. (main): V = e^{-rT} (2 pi)^{-d} int phi_T(-z) vhat(z) du on
 * Im z = delta, discretised on an N^d midpoint grid per axis as in Eq. (discr).
 * The N^d tensor of integrand values is put into tensor-train (matrix product
 * state) form by TT-cross with maxvol pivoting (Section IV.B) and contracted with
 * the quadrature weights (Section IV.A), at O(d N r^2) integrand evaluations.
 * The call on the maximum (not in the paper) is the sum of d such trains, one per
 * asset that can be the maximum.
 *
 * Conventions.
 *  - All arrays passed in are host memory owned by the caller and read only
 *    during the call.  Prices and diagnostics are written to caller-owned host
 *    memory.  The library owns all device memory it allocates; a caller may
 *    instead hand it a device workspace (tt_options.workspace).
 *  - Functions return a tt_status; tt_price_evaluate returns the worst status
 *    over the batch and never aborts the batch for one bad problem: a problem
 *    that fails validation or collapses numerically gets price NaN and its own
 *    status in tt_diag.
 *  - A handle is not thread-safe; all work runs on tt_options.cuda_stream.
 */
#ifndef TTPRICE_H
#define TTPRICE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tt_pricer tt_pricer; /* opaque, library-owned */

typedef enum {
  TT_OK = 0,
  TT_WARN_NOT_CONVERGED = 1, /* sweep cap reached before the stop rule held */
  TT_ERR_INVALID = -1,       /* bad argument or size */
  TT_ERR_NOT_PD = -2,        /* covariance failed an FP64 Cholesky (paper assumes PD, Sec. II.A) */
  TT_ERR_STRIP = -3,         /* damping outside the payoff transform's strip (Sec. III.C) */
  TT_ERR_CAPACITY = -4,      /* exceeds the sizes the handle was created for */
  TT_ERR_CUDA = -5,          /* a CUDA call failed */
  TT_ERR_NUMERIC = -6        /* fiber matrix of numerical rank 0, or a non-finite price */
} tt_status;

typedef enum { TT_MIN_CALL = 0, TT_MAX_CALL = 1 } tt_payoff;

/* TT_FP64: every step in FP64.
 * TT_MIXED: integrand values, elimination and maxvol in FP32 complex; the phase
 * and exponent arguments, the contraction and the interpolation solve in FP64
 * (refined from maxvol's FP32 inverse with FP64 residuals to the FP64 solution,
 * FP64 elimination when the refinement does not converge). */
typedef enum { TT_FP64 = 0, TT_MIXED = 1 } tt_precision;

/* Engine of the maxvol block product in the mixed path (Section IV.B cross step):
   FP32 FMA on the CUDA cores, or 3xTF32 tcgen05 MMAs with TMEM accumulators.
   Results agree to the mixed path's tolerance; speed depends on the rank. */
typedef enum { TT_ENGINE_AUTO = 0, TT_ENGINE_CUDA_CORES = 1, TT_ENGINE_TENSOR_CORES = 2 } tt_engine;

/* TT_METHOD_SINGLE_TRAIN: TT-cross of the product integrand phi_T(-z) vhat(z), its
 * train contracted with the weights.  TT_METHOD_TWO_TRAINS: the paper's bra-ket
 * form (Section IV, Eq. braket): the payoff transform vhat(z) and the
 * characteristic function phi_T(-z) are put into tensor-train form separately
 * (same rank cap; a fixed max_half_sweeps, default 3: left-to-right,
 * right-to-left, left-to-right, the train being the last one's cores; no
 * sum-based stop) and the two trains are contracted site by site,
 * E <- sum_i G^v_k(i)^T E G^phi_k(i), in FP64 in both precisions (TT_MIXED
 * runs the two crosses in FP32).  The two trains have their own bond
 * dimensions (tt_problem.max_rank and max_rank_phi, the paper's D_v and D_phi).
 * Needs max_rank <= 40 and the bracket's shared memory within the SM's
 * (max_n <= 1024 up to rank 32, about 512 at rank 40). */
typedef enum { TT_METHOD_SINGLE_TRAIN = 0, TT_METHOD_TWO_TRAINS = 1 } tt_method;

/* Per-class launch configuration (the autotuner's output): problems with
 * d_min <= d <= d_max, grid size n_grid (0: any), rank cap max_rank (0: any) and
 * payoff (a tt_payoff, or -1: either) run with these values instead of the
 * options' block_rows and rank_tol; the first matching class applies.  0 or a
 * non-positive value keeps the options' value.  A class's block_rows must lie
 * in [its problems' rank cap, tt_options.block_rows] (shared memory is sized for
 * the options' value); a problem whose rank cap exceeds it keeps the options'. */
typedef struct {
  int d_min, d_max;
  int n_grid;
  int max_rank;
  int payoff;
  int block_rows;
  double rank_tol;
} tt_class_tuning;

#define TT_MAX_CLASSES 64

typedef struct {
  int max_d;            /* largest number of assets                        (1..255)  */
  int max_n;            /* largest grid size N per axis                    (2..4096) */
  int max_rank;         /* largest TT rank                                 (1..64)   */
  int max_batch;        /* largest number of problems per evaluate call            */
  tt_precision precision;
  int max_half_sweeps;  /* 0 -> 8 (alternating left-to-right / right-to-left)       */
  double sweep_tol;     /* <= 0 -> 1e-6 (FP64) or 1e-4 (mixed): relative change of
                           the price estimate between half-sweeps that stops a job
                           (each path's accuracy target against the FP64 oracle)  */
  double rank_tol;      /* <= 0 -> 1e-8 (FP64) or 1e-6 (mixed): a column whose
                           elimination pivot is below rank_tol times the column's
                           largest entry is dropped (numerically dependent)        */
  double maxvol_tol;    /* <= 0 -> 0.05: maxvol stops when all |B_ij| <= 1 + tol  */
  int block_rows;       /* 0 -> 128: rows per elimination/maxvol block;
                           needs max_rank <= block_rows <= 256 - max_rank, and
                           block_rows <= 128 with TT_ENGINE_TENSOR_CORES (the
                           block product is one 128-row tensor-core tile)        */
  int engine;           /* tt_engine of the maxvol block product B = A P^{-1};
                           TT_ENGINE_AUTO picks CUDA cores up to max_rank 32 and
                           tensor cores above; TT_FP64 always uses CUDA cores    */
  int graph;            /* 1: tt_price_run replays a CUDA graph of its launches
                           (counter reset, TT-cross kernel, the bracket kernel
                           in the two-train form, finalize), captured
                           once per batch layout on a stream the pricer owns and
                           ordered after / before cuda_stream by events; 0: plain
                           launches on cuda_stream                               */
  int method;           /* tt_method (0: single train)                             */
  int device;           /* CUDA device ordinal                                     */
  void* cuda_stream;    /* cudaStream_t to run on; NULL = legacy default stream    */
  void* workspace;      /* optional device buffer of tt_workspace_bytes() bytes,
                           owned by the caller; NULL = the library allocates       */
  size_t workspace_bytes;
  const tt_class_tuning* classes; /* optional per-class block_rows / rank_tol, read
                           (copied) by tt_price_create; NULL = none              */
  int n_classes;        /* entries of classes (0..TT_MAX_CLASSES)                  */
  int pivot_io;         /* 1: keep every train's final pivots for tt_price_pivots
                           and accept tt_problem.warm_sets (device memory of
                           tt_pivot_record_entries() per train, twice); 0: neither */
} tt_options;

typedef struct {
  int d;                 /* number of assets                                       */
  const double* spot;    /* [d] S0_j > 0                                           */
  const double* cov;     /* [d*d] row-major annualised covariance, SPD             */
  double rate;           /* r                                                      */
  double maturity;       /* T > 0                                                  */
  double strike;         /* K > 0                                                  */
  int payoff;            /* tt_payoff                                              */
  const double* damping; /* [d] alpha_j.  Min-call: Im z_j = -alpha_j, needs
                            -alpha_j > 0 and sum_j -alpha_j > 1.  Max-call term j:
                            Im z_j = 1 + |alpha_j| and Im z_l = -|alpha_l| (l != j),
                            needs every alpha_l != 0                               */
  int n_grid;            /* N grid points per axis (midpoints of [-L, L])          */
  double trunc_L;        /* L > 0                                                  */
  int max_rank;          /* TT rank cap for this problem (<= tt_options.max_rank)  */
  unsigned long long seed; /* initial random pivots (SplitMix64), per problem       */
  int max_rank_phi;      /* two-train form only: bond dimension D_phi of the
                            characteristic function's train (0: max_rank); the
                            payoff transform's train takes max_rank (D_v).  Needs
                            max_rank * max_rank_phi <= 1024, else TT_ERR_CAPACITY */
  const unsigned short* warm_sets; /* optional warm start (needs pivot_io): initial
                            right index sets of TT-cross (Section IV.B starts from
                            column sets J_k, at random by default), for each train
                            of the problem in turn (1 or d terms, single-train
                            form), in the format tt_price_pivots writes: for
                            k = 1..d-1 a count c_k, then c_k distinct multi-indices
                            of grid points over axes k..d-1 (d-k entries each, each
                            < n_grid).  The first min(c_k, r_k) take the first slots
                            of bond k; the rest are drawn as usual.  NULL = none;
                            bad data gives TT_ERR_INVALID for the problem        */
} tt_problem;

typedef struct {
  int status;            /* tt_status of this problem                              */
  int half_sweeps;       /* largest number of half-sweeps over its trains          */
  int final_rank_max;    /* largest TT rank after rank reduction                   */
  int terms;             /* trains: 1 (min-call) or d (max-call), twice that in
                            the two-train form (a vhat and a phi train per term)  */
  long long evaluations; /* integrand evaluations, fiber entries counted once      */
  long long maxvol_swaps; /* row swaps made by maxvol, all cores and half-sweeps    */
  long long block_visits; /* maxvol block visits (one block product B = A P^{-1} each) */
  int fail_step;         /* for TT_ERR_NUMERIC: 1 fiber of rank 0, 2 singular pivot
                            block in maxvol, 3 singular interpolation solve,
                            4 non-finite estimate; 5 initial pivots not drawable;
                            6 a tensor-core block product did not complete (mixed);
                            8 (mixed) no half-sweep estimate of a train was
                            plausible (see 7) and the last one's share of the
                            price exceeds the sum of the spots; 9 (two-train
                            form) a singular pivot block or a non-finite value
                            in the bracket;
                            with TT_WARN_NOT_CONVERGED: 7 the mixed path reports an
                            earlier half-sweep's estimate of some train: the last one
                            moved by over 100x a plausible one before it, or was not
                            plausible itself, with an imaginary part above 1/4 of
                            its real part (the exact grid sum is real) or a share of
                            the price outside (0, sum of spots]; the reported one is
                            the latest plausible one                             */
  int maxvol_rollbacks;  /* cores whose maxvol returned to its last verified pivot set
                            after the working-precision pivot block became singular */
  double imag_part;      /* Im of the discrete sum; 0 up to the TT error           */
  double flops;          /* arithmetic of the elimination, maxvol, interpolation
                            and integrand steps, by formula: 24 per integrand
                            evaluation, 8 per complex multiply-add, 8 r^3/3 + 8 r'r
                            per interpolation solve (w = v S, then y P = w as an
                            elimination would count it, however it is solved)   */
  double est_discretization_err; /* estimated |grid price - integral| (absolute,
                            price units) from the Poisson-summation model of the
                            midpoint rule (Eq. discr): each axis aliases at rate
                            delta_j (|alpha_j| for the call on the maximum), a term
                            exp(-2 pi rate / eta) times the price, plus the cut
                            Gaussian tail exp(-T sigma_j^2 L^2 / 2) times the
                            price; an order-of-magnitude estimate (within a few
                            times where aliasing dominates, conservative where
                            the truncation does); NaN with a NaN price          */
} tt_diag;

/* Create a pricer for problems up to the given sizes on opt->device.  Allocates
 * all device memory the handle needs (unless opt->workspace is given).
 * Returns TT_OK, TT_ERR_INVALID or TT_ERR_CUDA; *out is NULL on failure. */
int tt_price_create(const tt_options* opt, tt_pricer** out);

/* Device bytes tt_price_create needs for these options (for a caller-owned
 * workspace).  0 if the options are invalid. */
size_t tt_workspace_bytes(const tt_options* opt);

/* Price count (<= max_batch) problems.  Blocking: returns after prices[] and
 * diag[] (nullable) are written.  Equivalent to tt_price_prepare +
 * tt_price_run + tt_price_results. */
int tt_price_evaluate(tt_pricer* h, const tt_problem* probs, int count, double* prices,
                      tt_diag* diag);

/* Validate and derive the per-train parameters on the host (FP64), and copy them
 * to the device (one asynchronous host-to-device copy on the handle's stream).
 * Per-problem validation failures are recorded, not returned as errors; the
 * return value is TT_ERR_INVALID/CAPACITY/CUDA only for batch-level failures. */
int tt_price_prepare(tt_pricer* h, const tt_problem* probs, int count);

/* Launch the pricing kernels for the prepared batch on the handle's stream and
 * return without waiting.  Can be repeated (the batch stays resident). */
int tt_price_run(tt_pricer* h);

/* Copy the results of the last run to the host, wait for them, and write
 * prices[count] and diag[count] (nullable).  Returns the worst status. */
int tt_price_results(tt_pricer* h, double* prices, tt_diag* diag);

/* Bytes the last tt_price_prepare copied host-to-device and the last
 * tt_price_results copied device-to-host (for end-to-end accounting). */
int tt_price_transfer_bytes(const tt_pricer* h, size_t* h2d, size_t* d2h);

/* Allocation-free pricing, for callers that may not allocate memory in the
 * call: code running where an allocation can fail or stall (a latency-bound
 * quote loop, a plugin inside a host application that owns all device memory,
 * a process whose memory budget is fixed up front).  The paper has no
 * counterpart; it is a deployment aid.
 *
 * Prices count <= TT_STATIC_MAX_BATCH problems, each with d <= TT_STATIC_MAX_D,
 * n_grid <= TT_STATIC_MAX_N and max_rank <= TT_STATIC_MAX_RANK, with the default
 * tolerances of tt_options, on the current CUDA device and the given stream
 * (NULL = legacy default stream).  Same results as tt_price_evaluate with those
 * options.  Blocking, like tt_price_evaluate.
 *  - Memory: no cudaMalloc/cudaFree/host allocation.  Device scratch is one
 *    file-scope array of TT_STATIC_SCRATCH_BYTES that every GPU loading this
 *    library holds until the process exits; host staging is file-scope arrays.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and sets kernel attributes; make that first call
 *    before any stream capture on that device.
 *  - Every call reuses the same arrays and overwrites the previous call's
 *    contents.  Calls that overlap (other threads, other streams) race; callers
 *    must serialise them.
 *  - Returns TT_ERR_CAPACITY if count exceeds TT_STATIC_MAX_BATCH; a problem
 *    beyond the size limits gets TT_ERR_CAPACITY in its tt_diag and a NaN price. */
#define TT_STATIC_MAX_BATCH 64
#define TT_STATIC_MAX_D 8
#define TT_STATIC_MAX_N 256
#define TT_STATIC_MAX_RANK 32
#define TT_STATIC_SCRATCH_BYTES (16u << 20)
int tt_price_evaluate_static(const tt_problem* probs, int count, int precision, void* cuda_stream,
                             double* prices, tt_diag* diag);

/* The final right index sets of problem `problem` of the last run (every train
 * in turn, in the warm_sets format above; after the last right-to-left
 * half-sweep, or the initial sets when none ran), for warm-starting a later
 * solve of a nearby problem.  Needs tt_options.pivot_io.  Copies to the host
 * and waits.  Returns the number of entries written (<= cap), or a negative
 * tt_status (TT_ERR_CAPACITY when cap is too small). */
int tt_price_pivots(tt_pricer* h, int problem, unsigned short* out, size_t cap);

/* Entries of one train's pivot record for problems up to max_d assets and rank
 * max_rank: (max_d - 1) counts and max_rank (d - k) indices per bond k. */
size_t tt_pivot_record_entries(int max_d, int max_rank);

/* Release everything the handle owns.  NULL-safe. */
void tt_price_destroy(tt_pricer* h);

/* Static text for a status code. */
const char* tt_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* TTPRICE_H */
