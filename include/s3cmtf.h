/*
 * s3cmtf.h -- C ABI of the GB300 (sm_103a) implementation of the S3CMTF hot path:
 * the per-nonzero SGD epoch of sparse coupled Tucker matrix-tensor factorisation
 * (Choi, Jang, Kang: "Fast, Accurate, and Scalable Method for Sparse Coupled
 * Matrix-Tensor Factorization", Section 3).
 *
 * Model (Section 2.2, Eq. (4); Section 2.3, Definition 1):
 *   x~_alpha = G x {u}_alpha = sum_j g_j prod_n u^(n)_{i_n j_n}        (tensor entry)
 *   y~_beta  = u^(c)_{j1} . v_{j2}                                      (coupled entry)
 * Objective (Eq. (7) and the per-entry sums after it):
 *   f = 1/2 sum_alpha [ e_alpha^2 + lambda_reg/|Omega| ||G||^2
 *                       + lambda_reg sum_n ||u^(n)_{i_n}||^2 / |Omega^{n,i_n}| ]
 *     + sum_m lambda_m/2 sum_beta [ e_beta^2 + lambda_reg/|Omega_Y^{2,j2}| ||v_{j2}||^2 ]
 * Per-entry gradients: Eq. (8).  Epoch: Algorithm 1 (with compute_gradient of
 * Algorithm 2/3), learning rate eta_t = eta_0 / (1 + mu t).
 *
 * Conventions for every call
 *   - Indices are 0-based int32.  Tensors are given structure-of-arrays: idx[n] points
 *     to the n-th index of every entry.
 *   - Factor matrices are dense row-major (I_n x J_n, K_m x J_c); the core is dense
 *     J_1 x ... x J_N with the last mode fastest.  All parameter buffers the caller
 *     passes are FP32 and unpadded.
 *   - "device" pointers are CUDA device (or managed) memory of the context's device;
 *     "host" pointers are ordinary (preferably pinned) host memory.
 *   - Inputs are owned by the caller and only read during the call.  The library keeps
 *     its own copies; nothing it allocates is handed to the caller.
 *   - All device work is ordered on the stream given to s3_init.  Calls that return a
 *     scalar to the host (s3_loss, s3_rmse) synchronise that stream; the others only
 *     enqueue work, except where stated.
 *   - Every call returns S3_OK or a negative status.  Invalid arguments and out-of-range
 *     indices are detected before any parameter is read with them: on the host for every
 *     array the library copies in (s3_init, s3_set_test, host-pointer s3_rmse), and by a
 *     check inside the kernel for the index arrays that stay in the caller's device memory
 *     (s3_predict, device-pointer s3_rmse, s3_rmse_noalloc): such an entry reads nothing and
 *     the call returns S3_ERR_INDEX.  No input can make a kernel fault.  After S3_ERR_CUDA
 *     the context is marked failed and every later call returns S3_ERR_STATE;
 *     s3_last_error() gives the text of the last error.
 */
#ifndef S3CMTF_H_
#define S3CMTF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct s3_ctx s3_ctx;  /* opaque, owned by the library */

enum {
    S3_OK = 0,
    S3_ERR_ARG = -1,       /* invalid argument, shape or unsupported configuration */
    S3_ERR_INDEX = -2,     /* an index outside its mode's range */
    S3_ERR_OOM = -3,       /* device or host allocation failed */
    S3_ERR_CUDA = -4,      /* a CUDA runtime error; the context is unusable afterwards */
    S3_ERR_DIVERGED = -5,  /* a non-finite parameter or loss was produced */
    S3_ERR_STATE = -6      /* NULL, destroyed or failed context */
};

enum { S3_MINIBATCH = 0, S3_HOGWILD = 1 };         /* epoch modes */
enum { S3_FP32 = 0, S3_BF16 = 1 };                 /* precision forms */
enum { S3_ROW_SUM = 0, S3_ROW_MEAN = 1 };          /* row rule of a group step */

/* Observed tensor entries Omega_X with their values (Section 2.3, Definition 2). */
typedef struct {
    int n_modes;                 /* N, 3 or 4 */
    const int64_t* dims;         /* host [N]: I_1..I_N */
    int64_t nnz;                 /* |Omega_X| */
    const int32_t* const* idx;   /* host array of N pointers, each [nnz] (host or device) */
    const float* val;            /* [nnz] (host or device) */
} s3_coo_tensor;

/* Observed entries of a matrix Y (I_c x K) coupled to tensor mode coupled_mode
   (Definition 1); its factor is V (K x J_c). */
typedef struct {
    int coupled_mode;            /* c, 0-based tensor mode */
    int64_t rows;                /* I_c (must equal dims[c]) */
    int64_t cols;                /* K */
    int64_t nnz;                 /* |Omega_Y| */
    const int32_t* r;            /* [nnz] row index j1 in [0, I_c) */
    const int32_t* c;            /* [nnz] column index j2 in [0, K) */
    const float* val;            /* [nnz]; NULL means every stored entry is 1 */
} s3_coo_matrix;

/* Hyper-parameters (Section 4.1 "Parameters"; the GPU group rules are this library's). */
typedef struct {
    float lr0;          /* eta_0 */
    float mu;           /* decay: eta_t = eta_0 / (1 + mu t), t = 0-based epoch */
    float lambda_reg;   /* regularisation of factors and core */
    float lambda_m;     /* weight of the coupled-matrix terms */
    int batch;          /* minibatch size B (items of the visiting order per step) */
    float core_scale;   /* core step = eta_t * core_scale * (mean core gradient of a group) */
    int row_rule;       /* S3_ROW_SUM or S3_ROW_MEAN: a row takes the sum, or the mean, of
                           its gradients within one group (batch or HOGWILD tile) */
    int hog_tile;       /* HOGWILD: tensor entries per tile of the FP32 kernel.  Its CTAs have
                           T compute threads, T = 384 for 3-way tensors up to padded rank 16
                           and 256 otherwise; a 3-way tile holds at most T / 2 entries (two
                           threads per entry; tiles of up to T / 4 spread each entry over
                           four), a 4-way tile T.  0 = default: T / 2 for 3-way tensors up to
                           rank 20 (192 at rank 10), 64 above, 128 with cp = 1, T for 4-way.
                           The BF16 kernel takes tiles of 128 entries (fewer only when a
                           tile's slots would not fit in shared memory). */
    float hog_staleness;/* HOGWILD: gamma of the staleness-aware row step.  A row expected to
                           have kappa > gamma updates in flight at once (kappa = its
                           occurrences x entries in flight / |Omega|) takes its step scaled by
                           gamma / kappa; every other row takes the plain lock-free step.
                           0 = default 360 / (largest rank), i.e. 36 at rank 10 (a coupled
                           entry's step grows stiffer with the rank), and 2000 / (largest rank)
                           in the non-negative form; < 0 disables the scaling. */
    int hog_ctas;       /* HOGWILD: CTAs working at once (0 = default: on 3-way tensors, enough
                           for a budget of tensor entries in flight -- 29184 up to rank 10,
                           29184 (10 / J)^0.6 at a larger largest rank J, three quarters of that
                           in the non-negative form -- at most as many as fit on the GPU, the
                           same number in both precision forms; on 4-way tensors as many as
                           fit).  Fewer CTAs mean fewer stale updates in flight and less
                           throughput. */
    int mb_ctas;        /* minibatch: CTAs of its persistent cooperative launch (0 = one per
                           SM, at most as many as fit); fewer CTAs make its grid-wide
                           barriers cheaper, more hide more load latency */
    int cp;             /* 1: S3CMTF-CP (Section 4.2), the core is hyper-diagonal: only G_j..j
                           are parameters (every mode needs the same rank); core steps and the
                           core gradient keep the diagonal, s3_set_params zeroes the rest, and
                           the HOGWILD epoch runs an O(N J) per-entry kernel.  FP32 form. */
    int nonneg;         /* 1: non-negative factorisation by projected SGD (Section 5,
                           "Discovery", which fits it with the projected gradient method): every
                           step of either mode is followed by max(0, .) on each parameter it
                           changed (rows, core).  HOGWILD applies the projection with an
                           atomic max after each atomic add, so the last operation on every
                           touched value is a projection.  A step whose result is NaN is
                           projected to 0 (minibatch) or kept, if its sign bit is clear
                           (HOGWILD).  Both precisions, and S3CMTF-CP.  The initial core may
                           hold negative entries until its first step; the factors start
                           non-negative (U(0,1)).  0 = the plain method. */
    int grad_chunk;     /* s3_gradient: items of the visiting order per chunk of the gradient
                           pass (its row-gradient slots are sized by one chunk's events);
                           0 = default 4194304.  Deterministic for a given value; the
                           compensated sums are carried across chunks. */
    int hog_core_sync;  /* BF16 HOGWILD: tiles over which a CTA accumulates its tiles' core steps
                           (in tensor memory) before adding them to G, lock-free, and re-reading
                           the core; between two such points the CTA computes with its own BF16
                           copy of the core.  0 = default, by the padded rank: 1 up to 10, 2
                           up to 20, 4 above.  1 = the per-tile core step of the FP32 form. */
    int wait_limit_us;  /* how long a bounded wait inside an epoch kernel (the minibatch epoch's
                           grid barrier, the BF16 kernel's tensor-core hand-offs) may last before
                           the kernel gives up, records where, and the epoch returns S3_ERR_CUDA
                           (the context is then failed; the device stays usable).  0 = default
                           2000000 (2 s). */
    int64_t device_bytes_cap;  /* the most device memory the context may allocate (its layout,
                           parameters and scratch); an allocation beyond it fails with
                           S3_ERR_OOM as if the device were full.  0 = no cap. */
} s3_hparams;

/* Create a context on the current CUDA device.
 *   train        tensor entries to fit (values FP32)
 *   Y, n_coupled coupled matrices (n_coupled may be 0, then Y may be NULL); at most 8
 *   J            host [N] core dimensionalities J_n (1..32)
 *   hp           hyper-parameters (copied)
 *   seed         seeds the initial parameters (factors and coupled factors U(0,1); core
 *                N(0, 3^N / prod J)), drawn by a counter-based generator (splitmix64)
 *                and, when order is NULL, the visiting order
 *   order        NULL, or [nnz + sum of coupled nnz] int64: the visiting order of the
 *                union of items (item k < nnz is tensor entry k; then the entries of each
 *                coupled matrix in turn) -- Algorithm 1 visits them "in random order"
 *   device_ptrs  0: every array above is host memory; 1: idx/val/r/c/val/order are
 *                device memory
 *   stream       cudaStream_t to order all work on (NULL = legacy default stream)
 * The entries are validated (range, finiteness), reordered into the library's layout
 * (visiting order, grouped into minibatches and HOGWILD tiles, each group's row
 * occurrences sorted into segments) and uploaded once.  Blocks until the layout is built.
 * On failure *out may still receive a context in the failed state so that
 * s3_last_error() can explain the status; release it with s3_destroy().
 */
int s3_init(s3_ctx** out, const s3_coo_tensor* train, const s3_coo_matrix* Y, int n_coupled,
            const int* J, const s3_hparams* hp, uint64_t seed, const int64_t* order,
            int device_ptrs, void* stream);

/* One pass over all items at eta_t, t = the context's epoch counter, which then advances.
 *   mode       S3_MINIBATCH: consecutive groups of hp.batch items of the visiting order;
 *              every gradient of a group is taken at the group-start parameters, rows
 *              take -eta_t * (sum or mean) of their Eq. (8) gradients, the core takes
 *              -eta_t * core_scale * (mean of its Eq. (8) gradients); deterministic.
 *              S3_HOGWILD: the lock-free scheme of Section 3.3 on the GPU: tiles of the
 *              visiting order run concurrently, each reading the current rows, combining
 *              its gradients per row (row_rule) and adding the step atomically (rows with
 *              many updates in flight take the staleness-aware step of hp.hog_staleness);
 *              the core is updated lock-free too: each tile adds core_scale / W of the
 *              core step of its mean gradient (W = tiles in flight), so that one wave of
 *              tiles moves the core by one group step; not deterministic.
 *   precision  S3_FP32 (CUDA-core FP32), or S3_BF16 (tensor-core contraction with BF16
 *              operands and FP32 accumulation; FP32 master parameters and errors; HOGWILD
 *              mode, 3-way tensors, ranks up to 32, computed at rank 16, 20 or 32 (the
 *              last mode padded to 32 at rank 20) with zero padding; else S3_ERR_ARG).
 * With hp.nonneg = 1 every step of either mode is a projected step (see s3_hparams).
 * Returns S3_ERR_DIVERGED if a non-finite parameter appeared (the parameters are left as
 * they are).  Enqueues work and synchronises once at the end to read the flag. */
int s3_epoch(s3_ctx* ctx, int mode, int precision);

/* f of Eq. (7) at the current parameters (FP32 errors, compensated FP32 partial sums,
 * FP64 final reduction), and the RMSE over the train entries.  Either output may be
 * NULL.  Synchronises. */
int s3_loss(s3_ctx* ctx, double* f_out, double* train_rmse_out);

/* test RMSE of Section 4.1 over the given entries (no clipping).  test == NULL uses the
 * entries given to the last s3_set_test.  Host or device pointers per device_ptrs; host
 * indices are checked on the host, device indices by the kernel (S3_ERR_INDEX, no RMSE
 * written, when one lies outside its mode's range).  Synchronises. */
int s3_rmse(s3_ctx* ctx, const s3_coo_tensor* test, int device_ptrs, double* rmse_out);

/* Keep a copy of test entries on the device for s3_rmse(ctx, NULL, ...). */
int s3_set_test(s3_ctx* ctx, const s3_coo_tensor* test, int device_ptrs);

/* Predictions x~ (Eq. (4)) at n coordinates: idx = host array of N device pointers each
 * [n] (0-based int32); out = device [n] FP32, caller-owned.  An index outside [0, I_n)
 * is caught inside the kernel: that entry reads no parameter and gets NaN, and the call
 * returns S3_ERR_INDEX.  Synchronises (to read that check). */
int s3_predict(s3_ctx* ctx, const int32_t* const* idx, int64_t n, float* out);

/* Full gradient (Eq. (8) summed over all train and coupled entries, the adjoint of the
 * tensor pass) at the current parameters, written to caller-owned device buffers of the
 * parameter shapes: dG [prod J], dU[n] [I_n * J_n], dV[m] [K_m * J_c].
 *   w   NULL: the gradient of f (Eq. (7)): every tensor entry's data terms carry -e_alpha.
 *       Else device [nnz] FP32 weights in the train-entry order given to s3_init: entry
 *       alpha's data terms carry w_alpha in place of -e_alpha, i.e.
 *         dU^(n)_i = sum_{alpha: i_n = i} w_alpha p_n(alpha) + lambda_reg u^(n)_i,
 *         dG       = sum_alpha w_alpha a_1 o .. o a_N + lambda_reg G,
 *       with the coupled-matrix terms of Eq. (8) unchanged (w = -e gives the same result as
 *       NULL).  The weights are read during the call; the library keeps no reference.
 * Rows without observed entries get zero.  Deterministic (fixed-order segmented reductions
 * with compensated FP32 sums). */
int s3_gradient(s3_ctx* ctx, const float* w, float* dG, float* const* dU, float* const* dV);

/* Partitioned problems (one process per GPU; mode-1 rows split across the processes, each
 * with the tensor entries and coupled entries of its rows, every other parameter replicated).
 * s3_set_counts gives a context that holds one part the counts of the whole problem, which
 * the regularisation terms of Eq. (7) and Eq. (8) use:
 *   counts     host array of N + n_coupled pointers to host int64 arrays: for every tensor
 *              factor row |Omega^{n,i}| (the whole problem's tensor entries in that row), then
 *              for every coupled factor row |Omega_Y^{2,k}| (its coupled matrix's entries in
 *              that column)
 *   nnz_total  |Omega| of the whole problem
 * It replaces the counts the context took from its own entries (S3_ERR_ARG, changing
 * nothing, when a count is below the context's own or nnz_total below its nnz).  After it,
 * s3_gradient returns this part's share of the whole problem's gradient: summed over the
 * parts (an all-reduce) it is the whole gradient (Eq. (8) summed over every entry).  The
 * HOGWILD step scales are not changed; s3_loss then counts this part's errors with the
 * whole problem's regularisers.
 * s3_apply_gradient takes one step of the minibatch rule whose group is a whole epoch, from
 * the whole gradient (device buffers of the parameter shapes): rows u <- u - eta_t dU, coupled
 * rows likewise, the core G <- G - eta_t core_scale dG / |Omega| (|Omega| = nnz_total), then
 * the projection of the non-negative form; the epoch counter advances.  The same gradient
 * applied by every part leaves identical replicas, and the step equals s3_epoch(S3_MINIBATCH)
 * with one batch holding the whole problem.  Row rule S3_ROW_SUM only (else S3_ERR_ARG);
 * S3_ERR_DIVERGED if a parameter became non-finite.  Synchronises. */
int s3_set_counts(s3_ctx* ctx, const int64_t* const* counts, int64_t nnz_total);
int s3_apply_gradient(s3_ctx* ctx, const float* dG, const float* const* dU, const float* const* dV);

/* Copy the parameters out to / in from caller-owned device buffers (shapes as above).
 * Used for checkpoint/resume (with s3_set_epoch) and to inject parameters. */
int s3_get_params(s3_ctx* ctx, float* G, float* const* U, float* const* V);
int s3_set_params(s3_ctx* ctx, const float* G, const float* const* U, const float* const* V);

/* Epoch counter t used for eta_t (read and set; resume = set_params + set_epoch). */
int s3_get_epoch(s3_ctx* ctx, int64_t* t);
int s3_set_epoch(s3_ctx* ctx, int64_t t);

/* Replace the observed values (not the coordinates) from HOST memory: the tensor's
 * values in the order given to s3_init and each coupled matrix's values likewise
 * (y_val may be NULL when n_coupled is 0; an entry y_val[m] may be NULL to keep that
 * matrix).  The host-to-device copy into one staging array is enqueued on the stream now;
 * each of the library's layouts (minibatch, HOGWILD, BF16 HOGWILD, gradient and loss) gathers
 * the staged values into its own order when a call next reads it, on the same stream.  Host
 * buffers must stay valid until the stream reaches the copy. */
int s3_update_values(s3_ctx* ctx, const float* x_val, const float* const* y_val);

/* The final QR step of Algorithm 1 (Section 3.4): for every mode n the thin QR
 * U^(n) = Q^(n) R^(n) with diag(R^(n)) > 0, then U^(n) <- Q^(n), G <- G x_n R^(n), and every
 * coupled factor of mode n  V_m <- V_m R^(n)^T.  Predictions of the tensor and of the
 * coupled matrices are unchanged up to FP32 rounding.  On the device: CholeskyQR2 in FP64
 * (two Gram passes over U), deterministic.  Returns S3_ERR_ARG, changing nothing, when some
 * U^(n) has fewer rows than its rank or is numerically rank deficient (a diagonal entry of
 * R^(n) at most 1e-7 of the largest).  Synchronises. */
int s3_finalize_qr(s3_ctx* ctx);

/* Sizes: number of items in the visiting order, groups per epoch for each mode. */
int s3_info(s3_ctx* ctx, int64_t* n_union, int64_t* n_batches, int64_t* n_tiles);

/* The HOGWILD launch of a precision form (S3_FP32 or S3_BF16): persistent CTAs, tensor
 * entries per tile (ctas x tile = entries in flight, the staleness of the lock-free
 * scheme), dynamic shared memory per CTA and the CTAs that fit on one SM.  ctas = 0 for
 * S3_BF16 when the form is not available for this context.  Any output may be NULL.
 * Returns S3_ERR_ARG for another precision. */
int s3_hog_config(s3_ctx* ctx, int precision, int64_t* ctas, int64_t* tile, int64_t* smem_bytes,
                  int64_t* ctas_per_sm);

/* Measurement support.  s3_profile(ctx, 1) makes the library record CUDA events on its
 * stream around every launch of its dominant kernels and count every kernel it launches;
 * s3_profile(ctx, 0) stops; enabling again clears the counters.  s3_profile_read gives,
 * for a kernel family, the summed event time of its launches (ms, synchronises), the
 * number of its launches and the tensor entries they processed; family -1 gives the
 * number of kernel launches of every kind (ms and entries 0).  Families:
 *   S3_K_TENSOR_HOG (HOGWILD tensor pass), S3_K_TENSOR_MB (the minibatch epoch, one
 *   persistent launch),
 *   S3_K_TENSOR_GRAD (gradient tensor pass), S3_K_TENSOR_FWD (loss / RMSE / predict). */
enum { S3_K_ALL = -1, S3_K_TENSOR_HOG = 0, S3_K_TENSOR_MB = 1, S3_K_TENSOR_GRAD = 2,
       S3_K_TENSOR_FWD = 3 };
int s3_profile(s3_ctx* ctx, int enable);
int s3_profile_read(s3_ctx* ctx, int family, double* ms, int64_t* launches, int64_t* entries);

/* Measurement support: the FP32 CUDA-core roof of the current device, measured.  Every SM
 * runs 64 warps of 16 independent FMA chains each, once with scalar FFMA and once with the
 * packed two-lane FFMA2; each rate (TFLOP/s, 2 flop per lane-FMA) is the best of three
 * launches of about 0.2 s timed with CUDA events on a private stream.  sm_mhz receives the
 * device's nominal maximum SM clock.  No context needed; changes no device setting.  Any
 * output may be NULL. */
int s3_measure_fp32_peak(double* ffma_tflops, double* ffma2_tflops, double* sm_mhz);

/* Test RMSE without allocating: the same value as s3_rmse(ctx, test, 1, ...) for callers
 * that must not allocate device memory while they run -- a process whose memory pool or
 * caching allocator has reserved the whole device (a cudaMalloc would fail or fragment it),
 * a job held to a fixed device-memory budget that was accounted up front, or a serving loop
 * that cannot take the device-wide synchronisation a cudaMalloc or cudaFree may cause --
 * while s3_rmse may grow its reduction buffer with cudaMalloc.  The paper has no
 * counterpart.
 *   idx       host array of N device pointers, each [n] (0-based int32 coordinates)
 *   val       device [n] observed values
 *   n         at most 2,097,152; larger n returns S3_ERR_ARG before any device work (split
 *             the call)
 *   rmse_out  host; sqrt(sum (val - x~)^2 / n)
 * Its only scratch is one static device array of about 64 KiB compiled into the library
 * (every GPU that loads the library holds it until the process exits).  The context's device
 * must be current (S3_ERR_ARG otherwise).  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) and keeps it; make that first call before any stream
 * capture.  Calls share the array, which keeps the last call's contents: calls whose work
 * overlaps on the GPU (other host threads, other streams, other contexts on the same
 * device) race on it and must be serialised by the caller.  An index outside its mode's
 * range is caught inside the kernel and returns S3_ERR_INDEX.  Enqueues on the context's
 * stream and synchronises it. */
int s3_rmse_noalloc(s3_ctx* ctx, const int32_t* const* idx, const float* val, int64_t n,
                    double* rmse_out);

const char* s3_last_error(const s3_ctx* ctx);
void s3_destroy(s3_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* S3CMTF_H_ */
