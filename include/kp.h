/*
 * kp.h -- C ABI of the GB300 (sm_103a) cross-matrix Krylov projection solver
 * for the implicit log-density Fokker-Planck systems of
 * "Efficient Score Pre-computation for Diffusion Models via Cross-Matrix
 * Krylov Projection" (arXiv 2511.17634).
 *
 * One linear system per (image channel, timestep n):  A^n m^n = b^n  (Eq. 12),
 * the five-point discretisation of Sec. 2.3 (Eq. 11 and its coefficient
 * listing), with the lagged field m~ = m^{n-1} in the first-order term.
 *
 * Vectors.  A channel of H rows and W columns is N = H*W doubles in the
 * paper's y-fastest order (Eq. 14): element p = i*H + j with i in [0,W) the x
 * index (east = i+1) and j in [0,H) the y index (north = j+1).  Out-of-grid
 * neighbours are zero (zero padding, Sec. 2.3).
 *
 * Memory and ownership.  Every vector argument is a DEVICE pointer owned by
 * the caller (8-byte aligned, N contiguous doubles); arrays of such pointers
 * (`const double* const* b`) and arrays of kp_op descriptors are HOST arrays
 * that the library copies before the call returns.  The library owns its
 * seed-basis store and workspaces; they live until kp_destroy.
 *
 * Streams.  All work is enqueued on the context's CUDA stream and the calls
 * return before it finishes; read outputs after synchronising that stream.
 * One context serves one stream from one host thread at a time.
 *
 * Errors.  Every call returns a kp_status: KP_OK, or a negative code for an
 * API-level failure (then nothing was enqueued and kp_last_error() explains
 * it).  Per-system convergence is reported through kp_info (device array),
 * never as a return code.  No C++ exception crosses this interface.
 */
#ifndef KP_H
#define KP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KP_OK = 0,
  KP_NOT_CONVERGED = 1,   /* kp_info.status: maxit reached, best iterate returned */
  KP_BREAKDOWN = 2,       /* kp_info.status: non-finite residual (NaN/Inf input)  */
  KP_ERR_ARG = -1,        /* invalid argument (size, pointer, option)               */
  KP_ERR_CUDA = -2,       /* a CUDA runtime call failed                             */
  KP_ERR_OOM = -3,        /* device allocation failed                               */
  KP_ERR_NO_BASIS = -4,   /* project_targets: no basis stored for (seed, timestep)  */
  KP_ERR_TIMEOUT = -5,    /* reserved: a bounded device wait gave up                */
  KP_ERR_UNSUPPORTED = -6,/* valid request this build does not implement            */
  KP_ERR_TOO_LARGE = -7   /* kp_refine_static: request exceeds its fixed scratch     */
} kp_status;

typedef enum {
  KP_PREC_FP64 = 0,  /* everything in FP64 */
  KP_PREC_MIXED = 1  /* FP32 Krylov vectors and stencil inside iterative
                        refinement whose solution, operator coefficients and
                        true residual b - A x are double-float (a pair of FP32
                        values, about 48 bits, on the FP32 pipe; FP64 in and
                        out); FP64 Hessenberg and Givens; BF16 tensor-core
                        projection with FP32 accumulation */
} kp_precision;

typedef struct kp_ctx kp_ctx;

/* Context options.  Fill with kp_options_default() and change what you need. */
typedef struct {
  int max_seeds;     /* seed-basis slots in the store (>= 1)                     */
  int max_a;         /* basis vectors kept per slot: a of Sec. 3 (1..64)          */
  int max_n;         /* largest N = H*W any call will pass (<= 16384)             */
  int precision;     /* kp_precision                                              */
  int smem_vectors;  /* Krylov vectors held in shared memory per system; the rest
                        live in a device workspace (0 = choose automatically)      */
  int reorth;        /* 0: CGS2, two classical Gram-Schmidt passes every step;
                        1: second pass only when the first removed more than
                        half of the vector's norm (Daniel-Gragg-Kaufman-Stewart)  */
  int block_threads; /* threads per system for grids of <= 1024 points: 256 (4
                        points per thread), 128 (8), 64 (16); 0 = 128 with 4
                        blocks per SM (FP64) or 256 with 2 (mixed precision) */
  int blocks_per_sm; /* resident solver blocks per SM for grids of <= 1024
                        points (caps registers per thread and sizes the
                        shared-memory window): 256 threads: 2 or 3; 128: 2, 3
                        or 4; 64: 4; 0 = the default above (2 for an explicit
                        256 or 128, 4 for 64).  Mixed precision: 2 always.   */
  int cluster_size;  /* mixed precision, grids of 1025..16384 points: solve each
                        system on a cluster of this many CTAs (2, 4 or 8 of 256
                        threads, <= 2048 points per CTA; or 16 of 128 threads,
                        <= 1024 points per CTA -- a non-portable cluster size;
                        W divisible by it); 0 = clusters only above 4096 points
                        (one 512-thread block below), of 2, 4 or 8 CTAs      */
  int fixed_a;       /* basis dimension of the seed solves (Sec. 3: V_a^n spans
                        the a-dimensional Krylov space; Sec. 5.2 uses a = 20):
                        0 = the first restart cycle ends when the seed meets its
                        tolerance, so a' = min(max_a, steps to converge) vectors
                        are kept; 1 = the first cycle keeps taking Arnoldi steps
                        until it has exactly a = min(max_a, m) vectors (fewer
                        only at an exact breakdown or maxit), and its iterate is
                        the GMRES minimiser over that whole space            */
  int inner_digits;  /* mixed precision: each FP32 inner GMRES reduces its
                        residual estimate by 10^-inner_digits (or to half of
                        the outer tolerance, whichever is reached first) before
                        the iterative refinement recomputes the true
                        residual; 1..7, 0 = 5                                     */
  int cluster_blocks_per_sm; /* cluster solver (grids above 4096 points): resident
                        CTAs per SM, 1 or 2 (16-CTA clusters: 2 or 4); 0 = 2
                        (16-CTA clusters: 4) -- several systems share the SMs,
                        each with a smaller shared-memory window of Krylov
                        vectors                                                  */
} kp_options;

/* Operator of one system (Sec. 2.3): A(m~; g^2, dt, h, f).  `mtilde` is the
 * lagged field m~ (device, N doubles).  fx, fy are the drift components on
 * the grid (device, N doubles each) or NULL for f = 0, the paper's setting
 * (Sec. 5).  g2 = (g^n)^2. */
typedef struct {
  int H, W;
  double dt, g2, h;
  const double* mtilde;
  const double* fx;
  const double* fy;
} kp_op;

/* Per-system result, written to a device array by the solver calls. */
typedef struct {
  int iters;       /* Arnoldi steps (operator applications, residuals excluded) */
  int status;      /* 0 converged, KP_NOT_CONVERGED, KP_BREAKDOWN               */
  double rel_res;  /* ||b - A x||_2 / ||b||_2 of the returned x, in FP64        */
} kp_info;

void kp_options_default(kp_options* opt);

/* Create a context bound to `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream) on the current device.  Allocates the basis store. */
kp_status kp_create(kp_ctx** ctx, const kp_options* opt, void* cuda_stream);
kp_status kp_destroy(kp_ctx* ctx);
kp_status kp_set_stream(kp_ctx* ctx, void* cuda_stream);
/* Last error message of this context (static string storage of the context). */
const char* kp_last_error(kp_ctx* ctx);
/* Library version string, e.g. "kp 0.1 sm_103a". */
const char* kp_version(void);

/*
 * y_k = A_k x_k for k < nsys (Sec. 2.3, Eq. 11; matrix form Eq. 12-13).
 * ops[k] describes A_k; x[k], y[k] device vectors of N_k doubles.
 */
kp_status kp_apply(kp_ctx* ctx, int nsys, const kp_op* ops, const double* const* x,
                   double* const* y);

/*
 * b_k = m^{n-1}_k / dt - Div_h f  (Sec. 2.3, right-hand side of Eq. 11).
 * mprev[k] device vector; f taken from ops[k].fx/fy (NULL = 0).
 */
kp_status kp_rhs(kp_ctx* ctx, int nsys, const kp_op* ops, const double* const* mprev,
                 double* const* b);

/*
 * Phase 1 of Sec. 3: solve the seed systems A_k x_k = b_k with restarted
 * GMRES(m) (CGS2 Arnoldi, FP64 Givens least squares, true FP64 residual at
 * every restart) to ||b - A x|| <= tol ||b|| or maxit Arnoldi steps.
 * x[k] holds the initial guess on entry (zero for the paper's seed solve) and
 * the solution on return.  The first restart cycle's orthonormal basis
 * v_1..v_{a'+1} (v_1 = r0/||r0||) and Hessenberg matrix of every system are
 * kept in the context until the next kp_seed_solve, for kp_store_basis.
 * info: device array of nsys kp_info, or NULL.  1 <= m <= 64; the number of
 * kept vectors a' = min(max_a, steps of the first cycle), which is
 * min(max_a, m) with kp_options.fixed_a = 1 unless Arnoldi breaks down.
 */
kp_status kp_seed_solve(kp_ctx* ctx, int nsys, const kp_op* ops, const double* const* b,
                        double* const* x, double tol, int m, int maxit, kp_info* info);

/*
 * Keep the basis of system `sys` of the last kp_seed_solve as the basis
 * V_a^n of seed slot `seed_id` for timestep `timestep` (Sec. 3: one basis per
 * timestep), replacing what the slot held.  Also factors H_a (Givens QR)
 * once, so that each projection needs only a rotation and a triangular solve.
 */
kp_status kp_store_basis(kp_ctx* ctx, int seed_id, int timestep, int sys);

/*
 * Phase 2 of Sec. 3 for nt targets that share seed slot `seed_id`:
 *   c = V_a^T r_k,   alpha = H_a^{-1} c,   x_k <- x_k + V_a alpha
 * with H_a = V_a^T A_seed V_a from the seed's Arnoldi process.  r_k is the
 * target's right-hand side b_k (paper: x_k = 0 on entry, so x_k becomes the
 * initial guess V_a alpha) or the residual b_k - A_k x_k of a guess x_k.  If
 * H_a is numerically singular (Givens pivot < 1e-14 max|H_a|) and v_{a+1} was
 * kept, alpha minimises ||Hbar_a alpha - V_{a+1}^T r_k|| instead.
 * Returns KP_ERR_NO_BASIS if the slot holds no basis for `timestep`.
 * ops[k] only supplies H, W (checked against the stored basis).
 */
kp_status kp_project_targets(kp_ctx* ctx, int seed_id, int timestep, int nt,
                             const kp_op* ops, const double* const* r_or_b, double* const* x);

/* As kp_project_targets, with a seed slot per target (one launch). */
kp_status kp_project_targets_multi(kp_ctx* ctx, int timestep, int nt, const int* seed_ids,
                                   const kp_op* ops, const double* const* r_or_b,
                                   double* const* x);

/*
 * The refine step of Sec. 3 (end of Phase 2): GMRES(m) on the target's own
 * A_k from the initial guess in x[k] to ||b - A x|| <= tol ||b|| (FP64 true
 * residual), or maxit Arnoldi steps.  Same algorithm as kp_seed_solve
 * without keeping a basis.  info: device array of nsys kp_info, or NULL.
 */
kp_status kp_refine(kp_ctx* ctx, int nsys, const kp_op* ops, const double* const* b,
                    double* const* x, double tol, int m, int maxit, kp_info* info);

/*
 * kp_refine_static -- kp_refine for callers that cannot allocate device memory.
 * (The paper has no counterpart: this is an interface for embedding.)
 *
 * Who needs it: code that may not call cudaMalloc or any allocating routine
 * when it solves -- a host whose memory pool or arena owns the device memory,
 * a plugin that may allocate only at start-up, a latency-critical path that
 * must never reach the allocator.  kp_refine needs a kp_ctx, and kp_create
 * and the solver calls allocate; this call needs neither a context nor any
 * allocation (no cudaMalloc, cudaFree, pinned or library allocation).
 *
 * Same algorithm and arguments as kp_refine (GMRES(m), CGS2, FP64), on the
 * caller's `cuda_stream` (a cudaStream_t, NULL = legacy default stream).  Its
 * scratch -- the system descriptors and the Krylov vectors beyond the shared
 * memory window -- is one static device array of KP_STATIC_SCRATCH_BYTES in
 * the library, held on every GPU that loads the library until the process
 * exits.  The descriptors reach the array as kernel parameters of small
 * copy launches (256 per launch), so no host staging buffer is involved.
 * Every call reuses that array and leaves its own contents there; nothing in
 * it has to start at zero, because each call writes every descriptor and
 * Krylov vector before reading it.  Calls whose work overlaps on the GPU
 * (other streams, other host threads) race on the array: order them, e.g.
 * on one stream.  A call that fails after it has enqueued work can leave the
 * array in any state; the next call rewrites everything it reads.
 *
 * Launch shape: one 256-thread block per SM of the current device, fewer
 * when their Krylov vectors beyond shared memory would not fit the array;
 * each block solves systems k, k + blocks, ...
 *
 * Limits: nsys <= KP_STATIC_MAX_SYSTEMS, H*W <= KP_STATIC_MAX_N, and one
 * block's Krylov vectors beyond shared memory must fit the array (always
 * true for m <= 64 on a GB300); otherwise KP_ERR_TOO_LARGE and nothing is
 * enqueued.  The first call on each device resolves the array's device
 * address (cudaGetSymbolAddress, once per device, with that device current,
 * under a lock shared by all devices) and so loads the library's module
 * there; make that first call before any stream capture.
 */
#define KP_STATIC_MAX_SYSTEMS 4096
#define KP_STATIC_MAX_N 1024
#define KP_STATIC_SCRATCH_BYTES (22u * 1024u * 1024u)
kp_status kp_refine_static(int nsys, const kp_op* ops, const double* const* b, double* const* x,
                           double tol, int m, int maxit, kp_info* info, void* cuda_stream);

/*
 * The contraction of Sec. 3, Phase 2 on the tensor cores:
 *   C[t][i] = sum_{k<K} B[t][k] V[i][k]   for t < nt, i < nv,
 * i.e. c_t = V_a^T b_t for every target, with tcgen05 MMAs (BF16 inputs, FP32
 * accumulation in tensor memory).  V: device BF16 [nv][ldv] (nv <= 48),
 * B: device BF16 [nt][ldb], C: device FP32 [nt][ldc]; ldv, ldb multiples of
 * 8 elements and V, B 16-byte aligned (TMA); K <= ldv, ldb.  Asynchronous on
 * the context's stream.
 */
kp_status kp_project_gemm_bf16(kp_ctx* ctx, int nt, int nv, int K, const void* B, int ldb,
                               const void* V, int ldv, float* C, int ldc);

/* r_k = b_k - A_k x_k (FP64), e.g. the residual of an initial guess before
 * projecting it (Sec. 3, Phase 2 in residual form). */
kp_status kp_residual(kp_ctx* ctx, int nsys, const kp_op* ops, const double* const* b,
                      const double* const* x, double* const* r);

/* ------------------------------------------------------------------------
 * Learned initial guess (not in the paper): a 3x3 convolutional network with
 * zero padding and ReLU between layers, trained on the GPU with this
 * library's kernels -- every convolution, its input gradient and its weight
 * gradient is a tcgen05 GEMM over im2col operands (BF16 inputs, FP32
 * accumulation); biases, ReLU, MSE loss and Adam (FP32 master weights, BF16
 * copies) are elementwise kernels.  Activations are FP32 planes
 * [batch][channels][H*W] in the solver's vector order.
 * Parameters (flat FP32): for each layer l, W_l [c_{l+1}][c_l][3][3] (tap
 * (di,dj) at index (di+1)*3 + (dj+1), di along x/columns, dj along y/rows),
 * then b_l [c_{l+1}].
 * ------------------------------------------------------------------------ */
typedef struct kp_cnn kp_cnn;
/* channels[0..nlayers]: c_0 (inputs) ... c_L (outputs), each 1..32. */
kp_status kp_cnn_create(kp_ctx* ctx, int H, int W, int max_batch, int nlayers,
                        const int* channels, kp_cnn** cnn);
kp_status kp_cnn_destroy(kp_cnn* cnn);
int kp_cnn_num_params(const kp_cnn* cnn);
kp_status kp_cnn_set_params(kp_cnn* cnn, const float* host_params);   /* resets Adam state */
kp_status kp_cnn_get_params(kp_cnn* cnn, float* host_params);
/* Size the inference buffers (the implicit-GEMM path of kp_cnn_forward and
 * the learned march) for B images, independently of the training batch of
 * kp_cnn_create (about 2.7 MB per 128x128 image).  Waits for the context's
 * stream; KP_ERR_UNSUPPORTED for shapes without that path (more than 16
 * input or output channels, one layer). */
kp_status kp_cnn_set_inference_batch(kp_cnn* cnn, int B);
/* out (device [B][c_L][H*W]) = network(in (device [B][c_0][H*W])); B <= the
 * inference batch (max_batch until kp_cnn_set_inference_batch). */
kp_status kp_cnn_forward(kp_cnn* cnn, int B, const float* in, float* out);
/* Loss = mean over B*H*W of (out - target)^2 (c_L = 1); gradients of the loss
 * (device [num_params], may be NULL) and the loss (host, may be NULL). */
kp_status kp_cnn_gradients(kp_cnn* cnn, int B, const float* in, const float* target,
                           float* grads, double* loss);
/* Network input of the learned guess for B targets at timestep n (1..T),
 * tau = n/T, dt = 1/T: planes [the target's lagged field m_i^{n-1} (its image
 * carried to timestep n-1) as hi = bf16(m) and lo = bf16(256 (m - hi)), the
 * seed state m_seed^n as hi and lo, tau, 1 - tau, sin pi tau, cos pi tau,
 * the residual the step leaves at the image, r = m/dt - A(m) m (Sec. 2.3 at
 * g^2 = g2n, f = 0), divided by rho = ||r|| / sqrt(H W), as hi and lo] into
 * in (device [B][10][H*W] FP32), and rho into rho (device [B]); mprev,
 * seed: host arrays of B device pointers to FP64 planes.  (A field in one
 * BF16 plane keeps 8 significant bits, too few for the step's change; hi and
 * lo keep about 16.) */
kp_status kp_cnn_pack_inputs(kp_cnn* cnn, int B, const double* const* mprev, const double* const* seed,
                             int n, int T, double g2n, float* in, double* rho);
/* Training target of the learned guess: out_b = (a_b - b_b) * scale / rho_b
 * (rho NULL: / 1), e.g. (m_i^n - m_i^{n-1}) / (dt rho_b) with scale = 1/dt,
 * into out (device [B][H*W] FP32); a, b: host arrays of device FP64 planes;
 * rho: device [B] or NULL. */
kp_status kp_cnn_pack_target(kp_cnn* cnn, int B, const double* const* a, const double* const* b,
                             const double* rho, double scale, float* out);
/* x_b = base_b + scale * rho_b * delta_b (rho NULL: 1): the FP64 initial
 * guess m_i^{n-1} + dt rho_b * network output with scale = dt. */
kp_status kp_cnn_add_guess(kp_cnn* cnn, int B, const float* delta, const double* const* base,
                           const double* rho, double scale, double* const* x);
/* One Adam step (Kingma & Ba 2015) on that loss; t = 1, 2, ... */
kp_status kp_cnn_train_step(kp_cnn* cnn, int B, const float* in, const float* target, float lr,
                            float beta1, float beta2, float eps, int t, double* loss);

/* Measured FMA throughput of this GPU's FP64 and FP32 pipes in TFLOP/s (2
 * flops per FMA; eight independent chains per thread, every SM filled, timed
 * with CUDA events on the context's stream): the denominators of the
 * solvers' ALU roofline.  Waits for the stream; allocates a few KB. */
kp_status kp_measure_alu_peaks(kp_ctx* ctx, double* fp64_tflops, double* fp32_tflops);

/* Inspect a stored basis (tests, diagnostics).  a_out, has_next_out, host.
 * V (device, N*(a+1) doubles, column k = v_{k+1}) and Hbar (host, (a+1)*a
 * doubles column-major, unrotated) may be NULL. */
kp_status kp_basis_get(kp_ctx* ctx, int seed_id, int timestep, int* a_out, int* has_next_out,
                       double* V, double* Hbar);

/* ------------------------------------------------------------------------
 * Time march (Sec. 2.3 with Sec. 3 applied at every timestep n = 1..T).
 *
 * For each timestep, in one stream and (by default) one CUDA graph per
 * parity of n:
 *   seeds:   b = m^{n-1}/dt, GMRES(m_seed) from x0 = 0 to tol_seed with the
 *            first-cycle basis kept (Phase 1), basis stored per seed;
 *   targets: b = m^{n-1}/dt, initial guess per `mode` -- PROJECTED: the
 *            Galerkin projection onto the basis of the target's seed (Phase 2);
 *            PLAIN: x0 = 0; WARM: x0 = m^{n-1} -- then GMRES(m) to tol;
 *   m^{n-1} <- m^n.
 * f = 0 (the paper's setting, Sec. 5), dt = 1/T, h = 1/H per group, and
 * g2[n-1] = (g^n)^2.  Groups may have different grid sizes; all seeds run in
 * one launch and all targets in one launch.  The seed bases of a timestep
 * live in one set of nseed_total context slots; a plan rotates 2 sets (one
 * timestep per launch) or 2K sets (windows of K timesteps), so max_seeds must
 * be at least 2 x nseed_total, and 2K x nseed_total for a window of K.
 * ------------------------------------------------------------------------ */
typedef enum {
  KP_MARCH_PROJECTED = 0,   /* the paper: x0 = V_a H_a^{-1} V_a^T b (seed's H_a)          */
  KP_MARCH_PLAIN = 1,       /* x0 = 0                                                      */
  KP_MARCH_WARM = 2,        /* x0 = m^{n-1}                                                */
  KP_MARCH_GALERKIN = 3,    /* exact Galerkin with the target's own operator:
                               x0 = V_a (V_a^T A_i V_a)^{-1} V_a^T b.  FP64 plans: G in the
                               solver; mixed precision (grids <= 4096 points, max_a + 1 <=
                               48): G = G0(seed basis) + Q_i P^T, the target's coefficient
                               row times the basis products on the tensor cores (BF16,
                               FP32 accumulation), c = V^T b likewise                     */
  KP_MARCH_LEARNED = 4,     /* the learned guess projected in residual form: x_init =
                               m^{n-1} + dt rho net(m^{n-1}, m_seed^n, time, r / rho)
                               (inputs as in kp_cnn_pack_inputs), x0 = x_init +
                               V_a H_a^{-1} V_a^T (b - A x_init) (mixed precision; needs
                               kp_march_opts.cnn)                                          */
  KP_MARCH_LEARNED_ONLY = 5 /* x0 = x_init, the learned guess alone (for comparison)    */
} kp_march_mode;

/* Phase 1 (Sec. 3) seed solver of a march.  BiCGSTAB is the method the paper
 * names: the orthonormalised key vectors of its first sweep (r_0, then s_k
 * and r_k of every iteration, each kept if it adds a direction, up to max_a)
 * are the stored basis, and A_proj = V^T A_seed V is formed explicitly and
 * solved by LU per target.  maxit counts BiCGSTAB iterations; m_seed must be
 * >= 4 (it sizes the solver workspace).  FP64 plans, one Picard iteration. */
typedef enum {
  KP_SEED_GMRES = 0,        /* restarted GMRES(m_seed), first-cycle Arnoldi basis */
  KP_SEED_BICGSTAB = 1      /* BiCGSTAB (van der Vorst 1992), key-vector basis     */
} kp_seed_solver;

typedef struct {
  int H, W;
  int nseed, ntgt;
  double* m_seed;        /* device [nseed][H*W]: m^{n0} in, m^{n0+steps} out   */
  double* m_tgt;         /* device [ntgt][H*W]                                   */
  const int* tgt_seed;   /* host [ntgt]: seed (index within this group) per target */
  /* Seed cycling with subspace expansion (Sec. 5.2: a new seed every h images,
   * the subspace capped at a), optional: host [nseed] or NULL.  seed_prev[s]
   * is the seed (index within this group, < s) whose basis seed s extends, or
   * -1.  Every timestep, the basis that seed s serves its targets becomes its
   * own basis vectors followed by the predecessor's served basis,
   * orthonormalised, capped at max_a, with A_proj = V^T A_s V formed with seed
   * s's operator (dense slot, LU per target).  FP64 plans. */
  const int* seed_prev;
} kp_group;

typedef struct {
  int T;                 /* timesteps of the full march; dt = 1/T              */
  const double* g2;      /* host [T]: (g^n)^2                                   */
  int mode;              /* kp_march_mode                                        */
  double tol_seed, tol;  /* relative residuals for seeds and targets             */
  int m_seed, m, maxit;  /* restart lengths, Arnoldi-step cap per solve          */
  int use_graph;         /* capture each timestep in a CUDA graph (1) or not (0) */
  int window;            /* FP64 plans: timesteps per target launch K (work items
                            claimed dynamically across the window); 0 = automatic
                            (8, capped by max_seeds / (2 x seeds): a window needs
                            2K basis slot sets), 1 = one timestep per launch.
                            Mixed precision and cluster shapes always use 1.     */
  int target_blocks;     /* window mode: persistent target blocks; 0 = every
                            resident slot of the GPU                              */
  /* Score extraction and probability-flow embedding (end of Sec. 2.3 and Sec.
   * 4.1), fused into the target solves (FP64 plans only), both optional:
   * score: device, [T][targets][2][H*W] FP64 -- for timestep n (1-based) and
   *   every target, in group order and the caller's target order within a
   *   group, sx = (m_{i+1,j} - m_{i-1,j}) / (2h) then sy = (m_{i,j+1} -
   *   m_{i,j-1}) / (2h) of m^n, zero outside the grid; a run writes the
   *   timesteps it solves (and, for n0 >= 1, timestep n0 again from its
   *   starting state: the same values when that state is the previous
   *   run's result).
   * embed: device, [targets][2][H*W] FP64 state x, advanced at timestep n by
   *   x += -dt (g^{n-1})^2 / 2 * grad m^{n-1} ((g^0)^2 = (g^1)^2); the caller
   *   sets x^0 (zero in the paper).  Must be given with score.          */
  double* score;
  double* embed;
  int picard;            /* Picard iterations per timestep (Sec. 2.3): 0 or 1 = one
                            solve with m~ = m^{n-1}; K > 1 re-solves with m~ the
                            latest iterate, same right-hand side, warm start; the
                            stored seed basis is the first solve's.  FP64 plans. */
  int seed_solver;       /* kp_seed_solver: how Phase 1 (Sec. 3) solves the seeds */
  int wait_probe;        /* testing aid for the bounded device waits, 0 normally.
                            1 (window plans, K > 1): every target item waits for a
                            release of its system that never comes, so each wait
                            gives up after 2^14 polls; the next kp_march_run call
                            that waits for the GPU returns KP_ERR_TIMEOUT (the
                            states are then not trustworthy) and the context stays
                            usable. */
  int maxit_seed;        /* Arnoldi-step cap of the seed solves; 0 = maxit         */
  kp_cnn* cnn;           /* KP_MARCH_LEARNED / _ONLY: the network (channels 10 -> ... -> 1,
                            the march's H x W, created on this context); every
                            timestep runs it on all targets in passes of its
                            inference batch (kp_cnn_set_inference_batch) inside the
                            march's graph, reading its current weights.  Do not use
                            the network on other work while a run is in flight.
                            One grid size, GMRES seeds, one Picard iteration.   */
} kp_march_opts;

/* Per-timestep totals, filled on the host by kp_march_run. */
typedef struct {
  double seed_iters, tgt_iters, tgt_iters_max, not_converged, max_rel_res;
  double refine_flops, seed_flops, proj_flops;   /* flops of the algorithm: FP64, except */
  double refine_flops32;                         /* FP32 Krylov flops (mixed precision)  */
} kp_step_stats;

/* Summed device time per kernel class (event-timed mode, launches in
 * sequence): seed_ms = seed GMRES with the fused basis store; refine_ms =
 * target GMRES with the fused projection; proj_ms = the learned guess
 * (input packing, network, x_init) of the learned modes; step_ms = first to
 * last event. */
typedef struct {
  float seed_ms, store_ms, proj_ms, refine_ms, step_ms;
  int launches;          /* kernel launches of this library in the run         */
} kp_march_timing;

typedef struct kp_march_plan kp_march_plan;

/* Builds the plan: device state, descriptors and (if use_graph) the graphs.
 * The group arrays are read now; their device buffers are used by every run.
 * Errors: KP_ERR_ARG for bad sizes, pointers, options, seed indices or
 * predecessors (seed_prev[s] outside -1..s-1), or more seeds than max_seeds / 2
 * (max_seeds / (2K) limits the window K); KP_ERR_UNSUPPORTED for grids above
 * 4096 unknowns in several groups, and for Picard iterations, exact Galerkin,
 * score extraction, BiCGSTAB seeds or seed cycling outside the FP64 one-block
 * solver (BiCGSTAB also needs one Picard iteration and m_seed >= 4);
 * KP_ERR_CUDA / KP_ERR_OOM for failed allocations, copies or graph captures.
 * On error *plan is NULL and nothing is left allocated. */
kp_status kp_march_create(kp_ctx* ctx, int ngroups, const kp_group* groups,
                          const kp_march_opts* opt, kp_march_plan** plan);
/* Runs timesteps n0+1 .. n0+steps (0 <= n0, n0+steps <= T) from the states in
 * the groups' buffers and leaves the result there.  stats (host, [steps]) and
 * timing may be NULL; when either is given the call waits for the GPU.  With
 * timing != NULL each kernel is bracketed by CUDA events (no graph).
 * Errors: KP_ERR_ARG for timesteps outside 1..T; KP_ERR_CUDA for a failed
 * launch or copy; KP_ERR_TIMEOUT (reported by the first call that waits for
 * the GPU, i.e. one with stats or timing) when a window's bounded wait for a
 * system's previous timestep gave up -- the states are then not trustworthy. */
kp_status kp_march_run(kp_march_plan* plan, int n0, int steps, kp_step_stats* stats,
                       kp_march_timing* timing);
kp_status kp_march_destroy(kp_march_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* KP_H */
