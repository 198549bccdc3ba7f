/*
 * gcp.h -- C ABI of libgcp: batched GCP-CROWN bound propagation on one GB300.
 *
 * GCP-CROWN (Zhang et al., "General Cutting Planes for Bound-Propagation-Based
 * Neural Network Verification", arXiv 2208.05740) lower-bounds
 *     f* = min_{x in C} c^T f(x),  C = {x : x_lo <= x <= x_hi}        (Sec. 2, Eq. 1)
 * for a ReLU network under general cutting planes
 *     sum_i H^(i) x^(i) + G^(i) xhat^(i) + Q^(i) z^(i) <= d               (Sec. 3.1, Eq. 15)
 * by propagating nu^(L) = -c backwards through every layer with the closed
 * form of Theorem 3.1 (App. A, Lemma A.1), then optimising the duals
 * alpha (ReLU lower slopes), beta (neuron-split multipliers) and gamma
 * (general-cut multipliers) by projected gradient ascent (Sec. 3.1 after
 * Theorem 3.1; App. C.1).
 *
 * Conventions shared by every call
 *  - Every call returns a gcp_status; nothing throws or aborts across the ABI.
 *    On error the call leaves its outputs untouched and gcp_last_error()
 *    describes the failure.
 *  - Host arrays passed in are copied; the caller keeps ownership and may free
 *    them when the call returns. Output arrays are caller-allocated.
 *  - "rows": a batch of S subdomains and K spec rows has R = S*K rows ordered
 *    r = s*K + k. Each row has its own alpha, beta, gamma (one dual point per
 *    subdomain and spec row).
 *  - A context owns one CUDA device and one stream; calls on one context are
 *    serialised by an internal mutex (thread-safe), calls on different
 *    contexts are independent.
 *  - Device-side failures (a kernel's bounds check or error word) surface as
 *    GCP_EDEVICE with a message; CUDA runtime errors as GCP_ECUDA.
 */
#ifndef GCP_H_
#define GCP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GCP_API __attribute__((visibility("default")))
#else
#define GCP_API
#endif

typedef struct gcp_ctx gcp_ctx;
typedef int32_t gcp_status;

enum {
  GCP_OK = 0,
  GCP_PENDING = 1,      /* gcp_serve_poll: request still in flight */
  GCP_EINVAL = -1,      /* malformed argument (shape, index, sign, NaN) */
  GCP_ENOMEM = -2,      /* device or host allocation failed */
  GCP_ECUDA = -3,       /* CUDA runtime error */
  GCP_ETIMEOUT = -4,    /* a bounded wait expired */
  GCP_EBUDGET = -5,     /* request larger than the context's HBM budget */
  GCP_ENOTFOUND = -6,   /* unknown net / cut set / duals / ticket */
  GCP_EDEVICE = -7      /* a kernel reported an error word */
};

enum { GCP_DENSE = 0, GCP_CONV2D = 1 };
/* cut variable kinds: pre-activation x, post-activation xhat, ReLU indicator z (Eq. 15) */
enum { GCP_VAR_X = 0, GCP_VAR_XHAT = 1, GCP_VAR_Z = 2 };
/* arithmetic of the propagation chain */
enum { GCP_FP64 = 0, GCP_FP32 = 1, GCP_BF16 = 2 };
enum { GCP_PGA = 0, GCP_ADAM = 1 };

/* One affine layer x^(i) = W^(i) xhat^(i-1) + b^(i) (Sec. 2).
 * dense : W is [d_out, d_in] row-major.
 * conv2d: W is [c_out, c_in, k, k] (OIHW), cross-correlation with the given
 *         stride and zero padding; activations are CHW-flattened, so
 *         d_in = c_in*h_in*w_in and d_out = c_out*h_out*w_out.
 * b has d_out entries (per output element, CHW order for conv2d).
 * skip: 0 for a plain layer; s >= 1 adds the post-activation xhat^(s-1) of an
 *       earlier layer (s = 1: the input x; s = i: the layer's own input) to
 *       the layer's output, x^(i) = W^(i) xhat^(i-1) + b^(i) + S xhat^(s-1):
 *       the shortcut of a residual block (ResBlock of the residual CIFAR
 *       models, Sec. 4 / App. C.1). Each xhat feeds at most one skip. The
 *       skip's multiplier nu^(i) adds S^T nu^(i) to the coefficient of
 *       xhat^(s-1) in the backward pass (Theorem 3.1 with S as one more
 *       linear map).
 * shortcut: NULL for the identity (S = I, needs d_{s-1} = d_out), else the
 *       projection S as a layer of its own (dense, or conv2d such as a 1x1
 *       stride-2 convolution; dense on the last layer) with d_in = d_{s-1},
 *       d_out = this layer's d_out, b = NULL (b^(i) carries the sum's bias),
 *       skip 0 and no shortcut. Read during gcp_init_net only.
 * Zero-initialise the struct to leave skip and shortcut off. */
typedef struct gcp_layer_desc {
  int32_t kind;
  int32_t d_in, d_out;
  int32_t c_in, h_in, w_in, c_out, h_out, w_out, k, stride, pad;
  const double* W;
  const double* b;
  int32_t skip;
  const struct gcp_layer_desc* shortcut;
} gcp_layer_desc;

/* Branch-and-bound subdomains as neuron split sets (App. B), CSR by
 * subdomain: subdomain s owns entries split_ptr[s] .. split_ptr[s+1]-1.
 * split_layer in 1..L-1, split_index < d_layer, split_sign +1 for the branch
 * x >= 0 and -1 for x <= 0. A split is the cut row -x <= 0 (resp. x <= 0) with
 * its own multiplier beta (Sec. 3.1, beta-CROWN as a special case) and clamps
 * the neuron's bound l := max(l,0) (resp. u := min(u,0)). */
typedef struct {
  int32_t n_sub;
  const int32_t* split_ptr;
  const int16_t* split_layer;
  const int32_t* split_index;
  const int8_t* split_sign;
} gcp_subdomains;

/* Optimiser settings. iters: gradient-ascent steps. optimizer: GCP_PGA
 * (x <- proj(x + lr*grad)) or GCP_ADAM (App. C.1; moments 0.9/0.999, eps 1e-8).
 * Learning rate at step t is lr * lr_decay^t. prec: chain arithmetic
 * (GCP_FP64 needs duals created with GCP_FP64; GCP_FP32 / GCP_BF16 need
 * GCP_FP32 duals). certify != 0: also run the FP64 outward-rounded
 * certification pass at the final duals.
 * opt_pi != 0: also optimise the ReLU duals pi (and gamma_r = C - pi) of every
 * unstable neuron directly, as App. A's closing remark suggests, instead of
 * Lemma A.1's closed form: pi = theta * [nuhat]_+ with theta in [0, 1] per row
 * and neuron, stepped at lr_alpha; it starts at the closed form, or continues
 * from the theta the duals object already holds (an earlier opt_pi call or
 * gcp_duals_theta). The object keeps theta, and every later bound, gradient
 * and certification of it uses theta until gcp_duals_import or an
 * optimisation with opt_pi = 0. Zero-initialise to leave it off. */
typedef struct {
  int32_t iters, optimizer, prec, certify;
  double lr_alpha, lr_beta, lr_gamma, lr_decay;
  int32_t opt_pi;
} gcp_opt_params;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`. hbm_budget_bytes caps the device
 * memory this context allocates (0 = no cap); exceeding it yields GCP_EBUDGET.
 * *out receives the context (owned by the caller, freed by gcp_destroy). */
GCP_API gcp_status gcp_create(gcp_ctx** out, int32_t device, uint64_t hbm_budget_bytes);
/* Free every net, cut set, duals object and the serving loop of the context. */
GCP_API gcp_status gcp_destroy(gcp_ctx* ctx);
/* Message of the last failing call on this context (static storage of the
 * context; valid until the next call). Never NULL. */
GCP_API const char* gcp_last_error(const gcp_ctx* ctx);
/* Use `stream` (a cudaStream_t passed as void*, NULL = the context's own
 * stream) for subsequent work of this context. The caller keeps ownership. */
GCP_API gcp_status gcp_set_stream(gcp_ctx* ctx, void* stream);
/* Device bytes currently held by the context. */
GCP_API gcp_status gcp_mem_used(const gcp_ctx* ctx, uint64_t* bytes);

/* ---------------------------------------------------------- problem inputs */

/* Register a network, its input box and spec (Sec. 2): layers[0..n_layers-1]
 * are W^(1)..W^(L); x_lo/x_hi [d_0] the input box (x0 -/+ eps for the
 * L-infinity ball); spec_c [n_spec, d_L] row-major, the spec rows folded in as
 * the last linear layer (nu^(L) = -c); inter_lo/inter_hi: sound pre-activation
 * bounds of hidden layers 1..L-1 concatenated ([sum d_i], Sec. 2, "sound
 * pre-activation bounds"), lo <= hi elementwise. *net_id receives the id.
 * Errors: GCP_EINVAL for inconsistent shapes, lo > hi or non-finite values. */
GCP_API gcp_status gcp_init_net(gcp_ctx* ctx, const gcp_layer_desc* layers, int32_t n_layers,
                                const double* x_lo, const double* x_hi,
                                const double* spec_c, int32_t n_spec,
                                const double* inter_lo, const double* inter_hi, int32_t* net_id);

/* Append n_cuts general cutting planes (Eq. 15) to a cut set of net_id:
 *   sum_{e in row_ptr[c]..row_ptr[c+1]-1} coef[e] * var(layer[e], kind[e], index[e]) <= d[c]
 * layer 0 is the network input (kind must be GCP_VAR_X); layers 1..L-1 are
 * hidden with kind X, XHAT or Z. *cutset_id: -1 creates a new cut set (id
 * returned in it), otherwise cuts are appended to that set (append-only, the
 * way cuts arrive from a MIP solver while branch and bound runs, Sec. 3.2).
 * *first_cut receives the index of the first appended cut. Duals created
 * later see all cuts; existing duals objects keep the cut count they had.
 * Errors: GCP_EINVAL for bad indices/kinds/non-finite values,
 * GCP_ENOTFOUND for unknown ids. */
GCP_API gcp_status gcp_add_cuts(gcp_ctx* ctx, int32_t net_id, int32_t n_cuts, const int64_t* row_ptr,
                                const int16_t* layer, const int8_t* kind, const int32_t* index,
                                const double* coef, const double* d, int32_t* cutset_id,
                                int32_t* first_cut);

/* ------------------------------------------------------------------- duals */

/* Create device-resident state for a batch of subdomains of net_id under
 * cut set cutset_id (-1 = no cuts): the duals alpha [R, sum_i d_i] (hidden
 * neurons, layer-major columns), beta [R, max_splits], gamma [R, N], the
 * split sets, and the workspace of the chain. dual_prec: GCP_FP64 (duals and
 * chain in float64) or GCP_FP32 (float32 duals; chain FP32 or BF16).
 * Default initial duals: alpha = 1 where u >= -l else 0, beta = gamma = 0.
 * *duals receives an opaque handle owned by the context. */
GCP_API gcp_status gcp_duals_create(gcp_ctx* ctx, int32_t net_id, int32_t cutset_id,
                                    const gcp_subdomains* sub, int32_t dual_prec, void** duals);
/* One batch for several queries on the same network, evaluated in the same
 * launches (uneven batching): query q has cut set cutset_ids[q] (-1 = none)
 * and subdomains subs[q]; rows are query-major (query 0's rows first). The
 * batch's cuts are the queries' cut sets concatenated in query order, and
 * the multipliers of a query's rows stay 0 on the other queries' cuts
 * (exported as zeros), so every row's bound is the one it has alone up to
 * summation order. Duals and errors as gcp_duals_create. */
GCP_API gcp_status gcp_duals_create_multi(gcp_ctx* ctx, int32_t net_id, int32_t n_queries, const int32_t* cutset_ids,
                                          const gcp_subdomains* subs, int32_t dual_prec, void** duals);
/* Shape of a duals object: rows R, alpha columns sum_i d_i, max_splits, cuts N. */
GCP_API gcp_status gcp_duals_shape(gcp_ctx* ctx, void* duals, int64_t* rows, int64_t* n_alpha,
                                   int32_t* max_splits, int32_t* n_cuts);
/* Copy the duals to host arrays (row-major [R, *]); NULL skips a group. */
GCP_API gcp_status gcp_duals_export(gcp_ctx* ctx, void* duals, double* alpha, double* beta, double* gamma);
/* Set the duals from host arrays (row-major [R, *]); NULL restores that
 * group's default initial value. Values are used as given (no projection). */
GCP_API gcp_status gcp_duals_import(gcp_ctx* ctx, void* duals, const double* alpha, const double* beta,
                                   const double* gamma);
GCP_API gcp_status gcp_duals_free(gcp_ctx* ctx, void* duals);
/* The directly optimised ReLU duals theta (opt_pi, pi = theta * [nuhat]_+),
 * row-major [R, n_alpha] in alpha's layout. theta_out != NULL copies them out
 * (GCP_ENOTFOUND while the duals object uses the closed form); theta_in !=
 * NULL sets them (used as given) and switches the object to theta. */
GCP_API gcp_status gcp_duals_theta(gcp_ctx* ctx, void* duals, const double* theta_in, double* theta_out);

/* ------------------------------------------------------------------ bounds */

/* Evaluate g(alpha, beta, gamma) of Theorem 3.1 at the current duals for all
 * R rows in chain arithmetic `prec` -> out_bound [R]. certify != 0 also runs
 * the certification pass -> out_certified [R]: the Lagrangian of Eq. 16 at
 * the dual point reached, evaluated in float64 with outward rounding and every
 * rounding residual charged over the variables' boxes, hence a rigorous lower
 * bound of the subdomain's optimum given sound intermediate bounds and valid
 * cuts (weak duality, App. A). out_certified may be NULL when certify == 0. */
GCP_API gcp_status gcp_bound_batch(gcp_ctx* ctx, void* duals, int32_t prec, int32_t certify,
                                   double* out_bound, double* out_certified);

/* Bound and its gradient d g / d(alpha, beta, gamma) at the current duals
 * (reverse mode of Theorem 3.1, computed by the adjoint kernels); outputs in
 * the export layouts. Any output may be NULL. */
GCP_API gcp_status gcp_grad_batch(gcp_ctx* ctx, void* duals, int32_t prec, double* out_bound,
                                  double* g_alpha, double* g_beta, double* g_gamma);

/* Run p->iters projected ascent steps on the duals in place (Sec. 3.1; App.
 * C.1), then evaluate at the final duals: out_bound [R] in p->prec; with
 * p->certify, out_certified [R] (FP64, outward rounded) and out_err_vs_fp64
 * [R] = |out_bound - out_certified|. Either of the last two may be NULL. */
GCP_API gcp_status gcp_optimize_batch(gcp_ctx* ctx, void* duals, const gcp_opt_params* p,
                                      double* out_bound, double* out_certified, double* out_err_vs_fp64);

/* The branching neuron of every subdomain of a batch at its current duals,
 * for a branch-and-bound loop (Sec. 3.2, App. B: a subdomain that is not
 * verified is split on one more unstable ReLU). One evaluation in chain `prec`
 * (GCP_FP32 or GCP_BF16; float duals) gives nuhat; over the root-unstable
 * neurons the subdomain has not split, the pick maximises
 * w_j * sum over the subdomain's spec rows of [nuhat_j]_+ with
 * w_j = -l_j u_j / (u_j - l_j): the part of the bound that the triangle
 * relaxation's intercept costs at neuron j (without cuts Lemma A.1 gives
 * pi* = u C / (u - l) and the term l pi* = -w_j C, C = [nuhat]_+), which a
 * split removes -- the intercept score of BaBSR (Bunel et al., 2020). Ties go
 * to the lower layer, then the lower index. layer[n_sub], index[n_sub]
 * (host) receive the pick, or -1 when every score is zero. */
GCP_API gcp_status gcp_branch_picks(gcp_ctx* ctx, void* duals, int32_t prec, int32_t* layer, int32_t* index);

/* Root intermediate bounds l, u of every hidden pre-activation (the sound
 * bounds Sec. 2 assumes, used by gcp_init_net), computed by this library's own
 * bound propagation, layer by layer. Hidden layer 1: the interval image of the
 * box under W^(1) x + b^(1), every product and sum rounded outwards on the host.
 * Hidden layer i > 1: the network truncated after the linear map of layer i,
 * with the spec rows +e_j and -e_j over its pre-activations, is bounded with
 * the already computed bounds of the layers below (at most 512 neurons per
 * batch): l_j = g(+e_j), u_j = -g(-e_j), each the FP64 outward-rounded
 * certified value, so the bounds are sound in any chain precision.
 * p == NULL: one evaluation at the default slopes (CROWN bounds). Otherwise
 * p->iters ascent steps on the slopes of every such row in the chain p->prec
 * (GCP_FP32 or GCP_BF16) with p's optimiser and rates (alpha-CROWN bounds);
 * p->certify is ignored (always on). layers / x_lo / x_hi as gcp_init_net
 * (n_layers >= 2; the last layer is not bounded). inter_lo / inter_hi: host,
 * caller-owned, sum of d_1 .. d_{L-1} doubles each (hidden layers in order);
 * untouched on error. Errors: GCP_EINVAL (shapes, null arguments, non-finite
 * bounds), and those of gcp_init_net / gcp_bound_batch / gcp_optimize_batch.
 * Temporary networks and duals are freed before returning. */
GCP_API gcp_status gcp_intermediate_bounds(gcp_ctx* ctx, const gcp_layer_desc* layers, int32_t n_layers,
                                           const double* x_lo, const double* x_hi, const gcp_opt_params* p,
                                           double* inter_lo, double* inter_hi);
/* The same with cutting planes (Eq. 15) in the propagation: hidden layer i's
 * bounds take every cut whose variables all lie in layers 0 .. i-1 (the
 * truncated network has them) with its multiplier gamma optimised together
 * with the slopes. With p == NULL (gamma = 0) the result is
 * gcp_intermediate_bounds'. The cuts must hold for every input of the box
 * (for example cuts of the root MIP, Sec. 3.2): root bounds are bounds over
 * the whole box. Cut arrays as in gcp_add_cuts (layer 0 = the input, kind
 * GCP_VAR_X there). Errors as gcp_intermediate_bounds and gcp_add_cuts. */
GCP_API gcp_status gcp_intermediate_bounds_cuts(gcp_ctx* ctx, const gcp_layer_desc* layers, int32_t n_layers,
                                                const double* x_lo, const double* x_hi, const gcp_opt_params* p,
                                                int32_t n_cuts, const int64_t* row_ptr, const int16_t* layer,
                                                const int8_t* kind, const int32_t* index, const double* coef,
                                                const double* d, double* inter_lo, double* inter_hi);

/* Branch and bound over ReLU splits (Sec. 3.2, App. B) with this library's
 * bounding: proves that every spec row of the network is positive over the
 * input box. Starting from the root (no splits), each round bounds up to
 * `batch` pending subdomains in one batch (p->iters ascent steps, then the FP64
 * certification; p->certify is forced on); when more are pending, the easiest
 * ones (largest lower bound) go first, the order of Sec. 3.2. A subdomain whose
 * certified bounds are all positive is verified; any other is split into the
 * x >= 0 and x <= 0 children of one more neuron, which start from the
 * parent's duals. branching = 0 picks the neuron by its duals at the end of
 * the round (gcp_branch_picks' score, from the round's last evaluation; the
 * static order below where every score is zero); branching = 1 takes the not
 * yet split root-unstable neuron with the largest relaxation intercept
 * -l u / (u - l) (a static order). Cuts (cutset_id >= 0) hold in every subdomain (they are valid
 * at the root). Stops when nothing is pending (verified = 1), after
 * max_rounds rounds, when more than max_domains subdomains are pending, after
 * timeout_s seconds, or when a subdomain with every root-unstable neuron split
 * still has a non-positive bound (verified = 0 in all these cases: not proven).
 * min_bound: the smallest certified bound over the bounded leaves and the
 * pending subdomains' priorities. The result is written only on GCP_OK. */
typedef struct {
  int32_t batch;         /* subdomains bounded per round, at most */
  int32_t max_rounds;
  int64_t max_domains;
  double timeout_s;      /* <= 0: none */
  gcp_opt_params p;
  int32_t branching;     /* 0: by the duals (gcp_branch_picks), 1: static root intercept */
} gcp_bab_params;
typedef struct {
  int32_t verified;
  int32_t rounds;
  int64_t domains_bounded, domains_verified, domains_left;
  double min_bound;
  double time_ms;
} gcp_bab_result;
GCP_API gcp_status gcp_bab_verify(gcp_ctx* ctx, int32_t net_id, int32_t cutset_id, const gcp_bab_params* bp,
                                  gcp_bab_result* res);
/* Branch and bound label by label (Sec. 3.2: the easiest target label first,
 * its root bound closest to zero, so that harder labels come later). Every
 * spec row is bounded at the root (one batch, p->iters steps, certified);
 * rows already positive are verified; each other row gets a branch and bound
 * of its own (as gcp_bab_verify on that single row, with bp's limits per
 * label). label_order[n_spec] receives the order in which the labels were
 * settled (root-positive ones first), label_verified[n_spec] 1 (proved), 0
 * (not proved) or -1 (not attempted: stop_at_failure != 0 and an earlier
 * label failed). res sums rounds and domains over the root batch and the
 * labels; min_bound is the smallest certified bound reached; verified = every
 * label proved. */
GCP_API gcp_status gcp_bab_verify_labels(gcp_ctx* ctx, int32_t net_id, int32_t cutset_id, const gcp_bab_params* bp,
                                         int32_t stop_at_failure, int32_t* label_order, int32_t* label_verified,
                                         gcp_bab_result* res);

/* Device-pointer entry points behind the PyTorch autograd wrapper.
 * alpha/beta/gamma are float32 device arrays in the export layouts; they
 * replace the duals object's values (copied in). gcp_bound_device writes the
 * FP32/BF16 bound [R] to out (device). gcp_grad_device runs the adjoint with
 * the per-row seed grad_out [R] (device) and writes vector-Jacobian products
 * into g_alpha/g_beta/g_gamma (device, export layouts). Work is enqueued on
 * `stream` (cudaStream_t as void*; NULL = the context stream, which does not
 * synchronise with the legacy default stream -- pass cudaStreamLegacy to
 * order the work with it) and the call returns without synchronising. */
GCP_API gcp_status gcp_bound_device(gcp_ctx* ctx, void* duals, int32_t prec, const float* alpha,
                                    const float* beta, const float* gamma, float* out, void* stream);
GCP_API gcp_status gcp_grad_device(gcp_ctx* ctx, void* duals, int32_t prec, const float* alpha,
                                   const float* beta, const float* gamma, const float* grad_out,
                                   float* g_alpha, float* g_beta, float* g_gamma, void* stream);

/* ------------------------------------------------------- no-allocation bound */

/* The FP32 bound g(alpha) of dense ReLU networks without cuts or splits,
 * enqueued on `stream` with no device allocation at all. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory -- processes that reserve the whole GPU for their own memory
 * pool up front, so that any further cudaMalloc fails, and loops that cannot
 * afford the device-wide synchronisation cudaMalloc and cudaFree imply.
 *
 * Every argument is the caller's and stays the caller's: dims (host,
 * d_0..d_L); WT, bias, lo, hi, alpha (host arrays of L-1 device pointers,
 * entry i-1 for layer i): WT = W^(i) transposed, float [d_{i-1}, d_i];
 * bias [d_i]; lo/hi the pre-activation bounds of hidden layer i [d_i];
 * alpha [R, d_i]; x_lo/x_hi [d_0] the input box; y_last [K, d_{L-1}] =
 * -W^(L)^T c_k and cb [K] = c_k^T b^(L) for the K spec rows; out [R]
 * receives the bound of row r = s*K + k. All device arrays are float32.
 *
 * The chain's scratch (its coefficients, one layer's product and the
 * objective partials: 3*R*max(d_0..d_{L-1}) + R*sum_i ceil(d_i/32) floats
 * plus offsets) lives in one 32 MiB device array of the library that every
 * GPU loading the library holds until the process exits; a batch that needs
 * more returns GCP_EBUDGET. The first call on each device looks up that
 * array's address (once, with the device current): make the first call
 * before any stream capture. Every call uses the same array, so calls whose
 * work overlaps on the GPU race and corrupt each other's results; serialise
 * them (one stream, or events). Returns without synchronising; GCP_EINVAL
 * for bad shapes or a pointer that is not device memory. */
GCP_API gcp_status gcp_bound_dense_noalloc(int32_t n_layers, const int32_t* dims, const float* const* WT,
                                           const float* const* bias, const float* const* lo,
                                           const float* const* hi, const float* const* alpha,
                                           const float* x_lo, const float* x_hi, const float* y_last,
                                           const float* cb, int32_t K, int64_t R, float* out, void* stream);

/* ------------------------------------------------------------- self-test */

/* Not a step of the paper's method: runs one GEMM of the chain on the current
 * device, C[M, N] = A[M, K] * B[N, K]^T (row-major float host arrays, copied
 * in and out), through kind 0 = tcgen05 bf16 (operands rounded to bfloat16),
 * 1 = tcgen05 three-pass tf32, 2 = the SIMT float kernel. For tests. Returns
 * GCP_EINVAL for a shape the kernel does not take (tensor-core kinds need
 * K % 8 == 0 for bf16, K % 4 == 0 for tf32). */
GCP_API gcp_status gcp_selftest_gemm(int32_t kind, int64_t M, int32_t N, int32_t K, const float* A, const float* B,
                                     float* C);

/* Not a step of the paper's method: the float64 product of the certification
 * pass, C[M, N] = A[M, K] * B[N, K]^T (row-major double host arrays), on the
 * tensor cores by exact bf16 slices, as the certification runs it for dense
 * layers. Cabs[M, N] (float) and *cerr give its rigorous error bound:
 * |C - exact| <= *cerr * Cabs elementwise. A row holding a non-finite value
 * gives NaN in C and +inf in Cabs. GCP_EINVAL when K has no slice plan
 * (K % 8 != 0, or K above about 18,000) or the tensor cores are unavailable.
 * For tests. */
GCP_API gcp_status gcp_selftest_gemm_f64(int64_t M, int32_t N, int32_t K, const double* A, const double* B, double* C,
                                         float* Cabs, double* cerr);

/* --------------------------------------------------------------- profiling */

/* Launch accounting (process-wide, all contexts). Not a step of the paper's
 * method: instrumentation for measuring it. After gcp_profile_start every
 * kernel launch of the library is counted with its algorithmic flops and
 * bytes (the minimum the launch must compute and move, from its shapes);
 * launches whose kernel name starts with kernel_prefix ("*" = all, NULL or ""
 * = none) are also bracketed by CUDA events on their own stream. */
GCP_API gcp_status gcp_profile_start(const char* kernel_prefix);
GCP_API gcp_status gcp_profile_stop(void);
/* While profiling: every launch of the idempotent tensor-core GEMMs
 * ("gemm_tc_tf32x3", "gemm_tc_bf16": they recompute their output from inputs
 * they do not write) whose name starts with kernel_prefix is issued twice, in
 * the same stream, so that the extra device time of a step over the launch
 * count is the kernel's cost inside the stream, with no event between
 * launches (NULL or "" = none; gcp_profile_stop clears it). The results do
 * not change. */
GCP_API gcp_status gcp_profile_repeat(const char* kernel_prefix);
/* Totals since gcp_profile_start for the kernel called `name` (NULL = all):
 * launches, device time of the timed launches (ms), flops, bytes. Waits for
 * the timed launches to finish. */
GCP_API gcp_status gcp_profile_query(const char* name, int64_t* launches, double* total_ms, double* flops,
                                     double* bytes);
/* One line per kernel, "name launches timed_launches ms flops bytes\n", into
 * buf (cap bytes, NUL-terminated); GCP_EINVAL if truncated. */
GCP_API gcp_status gcp_profile_report(char* buf, int64_t cap);

/* ----------------------------------------------------------------- serving */

/* A verification query for continuous batching: its subdomains (copied),
 * the optimiser settings of every round, and the number of branch-and-bound
 * rounds. Each round after the first replaces every subdomain by one child
 * (one more split on a root-unstable neuron chosen by the request's seed, on
 * a random side; App. B) and warm-starts its duals from the parent. */
typedef struct {
  int32_t net_id, cutset_id, rounds;
  uint64_t seed;
  gcp_subdomains sub;
  gcp_opt_params p;
  /* 1: keep the last round's subdomains and duals on the host when the
   * request finishes, for gcp_serve_final (costs one device-to-host copy of
   * rows x (hidden neurons + splits + cuts) floats); 0: drop them. */
  int32_t keep_final;
} gcp_request;

/* Result of a finished request. certified (caller-allocated, >= rows of the
 * last round) receives the certified bounds of the last round; min_certified
 * the minimum over them; latency_ms = completion - submission;
 * max_err_vs_fp64 = max over rows |chain bound - certified bound|, and
 * max_rel_err_vs_fp64 the same divided by max(1, |certified bound|). */
typedef struct {
  gcp_status status;
  int32_t rows;
  double* certified;
  double min_certified;
  double latency_ms;
  double max_err_vs_fp64;
  double max_rel_err_vs_fp64;
} gcp_result;

/* The final state of a request submitted with keep_final = 1: the subdomains
 * of its last round (split CSR as in gcp_subdomains; App. B's children after
 * rounds - 1 branchings) and the duals at which its certified bounds were
 * computed (layouts of gcp_duals_export: alpha [rows, sum of hidden widths],
 * beta [rows, max_splits] with slot m = the m-th split of the row's
 * subdomain, gamma [rows, n_cuts] over the request's cut set). The ReLU duals
 * theta of an opt_pi request are not included. */
typedef struct {
  int32_t n_sub, rows, n_alpha, max_splits, n_cuts;
  int64_t n_split_entries;
  int32_t* split_ptr;    /* [n_sub + 1] */
  int16_t* split_layer;  /* [n_split_entries] */
  int32_t* split_index;  /* [n_split_entries] */
  int8_t* split_sign;    /* [n_split_entries] */
  float* alpha;          /* [rows, n_alpha] */
  float* beta;           /* [rows, max_splits] */
  float* gamma;          /* [rows, n_cuts] */
} gcp_final;

/* Start the serving loop: a host scheduler thread admits submitted requests
 * while at most max_inflight run and their estimated device memory fits the
 * context's budget, keeps each admitted request's duals on the device between
 * rounds, and every round evaluates the active requests of one network (and
 * optimiser schedule) in one merged batch with shared launches (as
 * gcp_duals_create_multi); groups of different networks run concurrently on
 * their own streams. Requests submitted meanwhile join at the next round;
 * memory is freed as requests finish. Results are certified (FP64). */
GCP_API gcp_status gcp_serve_start(gcp_ctx* ctx, int32_t max_inflight);
/* Enqueue a request; *ticket identifies it. GCP_EBUDGET if it can never fit. */
GCP_API gcp_status gcp_serve_submit(gcp_ctx* ctx, const gcp_request* req, uint64_t* ticket);
/* GCP_PENDING while in flight; otherwise fills *res and forgets the ticket. */
GCP_API gcp_status gcp_serve_poll(gcp_ctx* ctx, uint64_t ticket, gcp_result* res);
/* Like poll but waits up to timeout_ms (GCP_ETIMEOUT if still pending). */
GCP_API gcp_status gcp_serve_wait(gcp_ctx* ctx, uint64_t ticket, int32_t timeout_ms, gcp_result* res);
/* The final state of a finished keep_final request whose result has been
 * taken by gcp_serve_poll / gcp_serve_wait. The sizes in *out are always
 * filled; when every pointer of *out is non-NULL the arrays are copied into
 * those caller-allocated buffers and the state is forgotten (a second call
 * gives GCP_ENOTFOUND). With any pointer NULL only the sizes are written (a
 * size query). GCP_ENOTFOUND: unknown ticket, no keep_final, or not yet
 * taken; GCP_EINVAL: the request failed. */
GCP_API gcp_status gcp_serve_final(gcp_ctx* ctx, uint64_t ticket, gcp_final* out);
/* Stop accepting submissions, finish every submitted request, join the
 * scheduler thread and free the loop's streams. Unpolled results and kept
 * final states are dropped. */
GCP_API gcp_status gcp_serve_stop(gcp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GCP_H_ */
