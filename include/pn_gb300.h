/*
 * pn_gb300.h -- C ABI of the GB300 (sm_103a) staggered-grid P_N library.
 *
 * The library applies and solves the discrete real-valued P_N system of
 * Koerner, Portsmouth and Jakob, "P_N-Method for Multiple Scattering in
 * Participating Media" (EGSR 2018):
 *
 *     A u = Q,   A = T + C - S                  (section "Discretized RTE")
 *
 * one equation per real SH coefficient (l, m), l <= N, at its staggered
 * location (appendix "Final equation"; section "Precomputation",
 * Fig. staggeredgrid).  Row (l, m) at location p reads
 *
 *     sum_d sum_(l',m') A_d[(l,m),(l',m')] (u_(l',m')(p + h/2 e_d)
 *                                         - u_(l',m')(p - h/2 e_d)) / h
 *   + (sigma_t(p) - sigma_s(p) g^l) u_(l,m)(p)  =  Q_(l,m)(p)
 *
 * with A_d the transport couplings of the printed equations (coefficients
 * a..f, beta, delta of the appendix, with the denominator of a read as
 * (2l+3)(2l+1) and the m>0 x-term of L^{l-1,m-1} read with e^{l-1,-m+1}),
 * the scattering factor lambda_l p^{l,0} = g^l of a normalised
 * Henyey-Greenstein phase function, a unit-cube grid of R^3 cells (h = 1/R),
 * and the Dirichlet rule of section "Runtime": a reference to a location
 * outside the closed domain is dropped.
 *
 * Staggering (the paper defers it to StaRMAP): coefficient (l, m) lives on
 * cell faces along every axis on which its harmonic is odd and on cell
 * centres along the others:
 *     p_x = m mod 2 (m >= 0), (|m|+1) mod 2 (m < 0);  p_y = [m < 0];
 *     p_z = (l + |m|) mod 2.
 * Along an axis with p = 0 the unknowns are the R cell centres (i+1/2) h;
 * with p = 1 they are the R+1 faces i h (boundary faces included).
 *
 * Parameters are given at voxel centres; sigma_t is clamped below by
 * sigma_t_min (sections "Runtime" and "Nebulae"), sigma_s = albedo sigma_t,
 * and both are interpolated to a location as the mean of the adjacent voxel
 * centres that lie inside the domain.
 *
 * ---------------------------------------------------------------------------
 * Vector layout (every x, y, r, u argument): "padded coefficient-major".
 * A vector holds K = (N+1)^2 planes; plane p stores coefficient
 * k = plane_k[p] (k = l*l + l + m) of parity class plane_class[p]
 * (class = p_x + 2 p_y + 4 p_z); planes are grouped by class.  Element
 * (z, y, x) of plane p is at
 *     p * plane_stride + z * pitch_y + y * pitch_x + x
 * and is an unknown ("active") iff x < R + p_x, y < R + p_y, z < R + p_z
 * (PN_BC_PERIODIC_TEST: iff x, y, z < R).
 * Every other slot is padding: kernels never read it and write it as 0.
 * Query the numbers with pn_get_layout().  Element type: float (PN_F32) or
 * double (PN_F64); base pointers must be 16-byte aligned.
 *
 * Ownership: pn_create copies the medium; x/y/r/u buffers belong to the
 * caller (device memory unless a call says otherwise); scratch and Krylov
 * work vectors belong to the handle and are freed by pn_destroy.
 * Streams: every call is ordered on the caller's cudaStream_t (NULL = the
 * legacy default stream).  Calls that return a host scalar synchronise that
 * stream.  A handle must not be used from two host threads at once (it owns
 * a side stream and events that the FP32 operator forks to and joins from).
 * Errors: every call returns PN_OK (0) or a negative PN_ERR_* code and never
 * aborts; pn_last_error() gives a message for the handle's last failure.
 */
#ifndef PN_GB300_H
#define PN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PN_OK                 0
#define PN_ERR_ARG           -1  /* invalid argument (null, N > 7, R < 2, dtype, ...) */
#define PN_ERR_ALLOC         -2  /* device or host allocation failed */
#define PN_ERR_CUDA          -3  /* a CUDA runtime call or kernel launch failed */
#define PN_ERR_NOT_CONVERGED -4  /* solver hit max_iter; x holds the last iterate */
#define PN_ERR_BREAKDOWN     -5  /* Krylov breakdown (zero norm denominator) */
#define PN_ERR_NONFINITE     -6  /* NaN or Inf met in a residual or inner product */
#define PN_ERR_TIMEOUT       -7  /* a bounded device-side wait (grid barrier) ran out */
#define PN_ERR_UNSUPPORTED   -8  /* valid request this build does not implement */
#define PN_ERR_TOO_LARGE     -9  /* request exceeds a fixed capacity of the library */

#define PN_F32 0
#define PN_F64 1

#define PN_BC_VACUUM 0           /* Dirichlet: outside references dropped */
#define PN_BC_PERIODIC_TEST 1    /* every axis wraps; R slots per axis for every coefficient (a test
                                    mode for exact closed forms; 3D only; the generic operator
                                    kernel serves it, FP32 included; unstagger and the learned
                                    preconditioner refuse it) */

#define PN_Q_CENTRE_00      0    /* Q: R^3 field of Q^{0,0} at voxel centres */
#define PN_Q_CENTRE_MOMENTS 1    /* Q: K x R^3 centre moments, k-major */

#define PN_MAX_N 7
#define PN_MAX_K 64

typedef struct pn_handle pn_handle;
typedef struct pn_cnn pn_cnn;

/* Voxel-centre medium.  Arrays are indexed [z][y][x] (x fastest), R^3 each. */
typedef struct {
    const void* sigma_t;   /* extinction, R^3 (required) */
    const void* albedo;    /* single-scattering albedo field R^3, or NULL */
    double albedo_const;   /* used when albedo == NULL */
    double g;              /* Henyey-Greenstein mean cosine, |g| < 1 */
    const void* Q;         /* source, layout per q_mode; NULL means Q = 0 */
    int q_mode;            /* PN_Q_CENTRE_00 or PN_Q_CENTRE_MOMENTS */
    int dtype;             /* PN_F32 or PN_F64: element type of the arrays */
    int on_device;         /* 1: device pointers, 0: host pointers */
    double sigma_t_min;    /* sigma_t := max(sigma_t, sigma_t_min); >= 0 */
} pn_medium;

typedef struct {
    int N, K, R;
    int64_t pitch_x;       /* elements between rows (y) */
    int64_t pitch_y;       /* elements between slices (z) */
    int64_t plane_stride;  /* elements between planes */
    int64_t n_elems;       /* vector length = K * plane_stride */
    int64_t n_active;      /* number of unknowns (degrees of freedom) */
    int plane_k[PN_MAX_K];     /* coefficient index stored in plane p */
    int plane_class[PN_MAX_K]; /* parity class of plane p */
} pn_layout_info;

/*
 * Create a handle for the P_N system of order N (1..7) on R^3 cells.
 * Copies and preprocesses the medium (clamp, sigma_s, Q in padded layout) into
 * device buffers owned by the handle.  Synchronises `stream` before returning.
 * boundary is PN_BC_VACUUM or PN_BC_PERIODIC_TEST.  On failure *out is NULL and the message is
 * available from pn_last_error(NULL).
 */
int pn_create(pn_handle** out, int N, int R, const pn_medium* medium, int boundary, void* stream);

/*
 * Create a handle for the 2D reduction of the P_N system (section "2D
 * checkerboard": parameters, source and boundary independent of z, so every
 * coefficient with l + m odd vanishes and the z-derivatives drop out) on R^2
 * cells of the unit square, R in [2, 16384].  The medium's arrays are
 * indexed [y][x], R^2 each; a PN_Q_CENTRE_MOMENTS source holds one R^2 field
 * per coefficient with l + m even, in increasing k = l^2 + l + m.
 * The handle's layout (pn_get_layout): K = (N+1)(N+2)/2 planes, the parity
 * classes with pz = 0 (0..3), each plane one slice of R+1 rows of pitch_x
 * (pitch_y elements used, plane_stride = pitch_y rounded up to 32); plane_k
 * holds the 3D coefficient index k.  Every operator, vector, solver and
 * unstagger entry point accepts the handle (pn_unstagger then writes K x R^2
 * in the order of the coefficient list); the learned preconditioner
 * (pn_cnn_features, pn_cnn_targets, pn_cnn_output, pn_cnn_precondition,
 * PN_SOLVER_IR_FGMRES) is 3D only and returns PN_ERR_UNSUPPORTED.
 * Errors and ownership as for pn_create.
 */
int pn_create_2d(pn_handle** out, int N, int R, const pn_medium* medium, int boundary, void* stream);

/* Free every buffer the handle owns.  NULL is accepted. */
int pn_destroy(pn_handle* h);

/* Fill *out with the vector layout (host struct). */
int pn_get_layout(const pn_handle* h, pn_layout_info* out);

/* Message of the last failure on h (h == NULL: last pn_create failure). */
const char* pn_last_error(const pn_handle* h);

/*
 * y = A x  (the matrix-free staggered operator; Eq. "(T + C - S) u = A u").
 * x, y: device vectors of `dtype` in the padded layout; must not alias.
 * Inactive slots of x are ignored; inactive slots of y are written 0.
 * The first FP64 operator call on a 3D vacuum-boundary handle (pn_apply,
 * pn_apply_t, pn_residual or a solver's refinement residual) allocates the
 * per-class means of sigma_t and sigma_s at every slot (16 planes of FP64),
 * kept until pn_destroy.
 */
int pn_apply(pn_handle* h, const void* x, void* y, int dtype, void* stream);

/*
 * y = A^T x.  The transport part is skew-symmetric under the Dirichlet rule,
 * so A^T = (C - S) - T; needed by CG on the normal equations (section
 * "Runtime", the paper's solver).  Same arguments as pn_apply.
 */
int pn_apply_t(pn_handle* h, const void* x, void* y, int dtype, void* stream);

/*
 * r = Q - A x.  If rel_out is not NULL, *rel_out (host) receives
 * ||r||_2 / ||Q||_2 accumulated in FP64 and the stream is synchronised
 * (||Q|| = 0 gives ||r||_2).  x and r must not alias.
 */
int pn_residual(pn_handle* h, const void* x, void* r, double* rel_out, int dtype, void* stream);

/* *out (host) = sum_i x_i y_i over the whole padded vector, accumulated in
 * FP64 in a fixed order (deterministic).  Synchronises the stream. */
int pn_dot(pn_handle* h, const void* x, const void* y, double* out, int dtype, void* stream);

/* y = alpha x + beta y over the whole padded vector (device vectors). */
int pn_axpby(pn_handle* h, double alpha, const void* x, double beta, void* y, int dtype, void* stream);

#define PN_SOLVER_CGLS     0     /* CG on the normal equations (the paper) */
#define PN_SOLVER_GMRES    1     /* restarted GMRES(m) on A u = Q */
#define PN_SOLVER_IR_GMRES 2     /* FP64 iterative refinement, FP32 GMRES inner */
#define PN_SOLVER_IR_FGMRES 3    /* FP64 iterative refinement, FP32 flexible GMRES inner,
                                    right-preconditioned by the learned network opts->precond */

typedef struct {
    int solver;          /* PN_SOLVER_* */
    int precision;       /* CGLS/GMRES: PN_F32 or PN_F64 vectors; IR: ignored */
    double tol;          /* target ||Q - A u||_2 / ||Q||_2 (FP64, original system) */
    int max_iter;        /* cap on inner Krylov iterations (all restarts/outer steps) */
    int restart;         /* GMRES basis size m (1..200) */
    double inner_tol;    /* IR: relative reduction asked of each inner solve */
    int max_outer;       /* IR: cap on refinement steps */
    int check_every;     /* iterations between host convergence checks */
    int profile;         /* 1: time every kernel launch of the solve with CUDA
                            events on the solve's stream (see pn_profile_get) */
    int ortho;           /* GMRES orthogonalisation: PN_ORTHO_CGS2 (classical
                            Gram-Schmidt twice) or PN_ORTHO_CGS1 (once, norm of
                            the new vector by Pythagoras, half the traffic) */
    void* precond;       /* PN_SOLVER_IR_FGMRES: the pn_cnn network (c_in = K + 3,
                            c_out = K) of pn_cnn_precondition; R a multiple of 8 */
    int basis;           /* PN_SOLVER_IR_GMRES: element type of the stored Krylov basis,
                            PN_BASIS_F32 (default) or PN_BASIS_F16 (FP16 values of
                            sqrt(n) v, FP32 arithmetic, one Gram-Schmidt pass,
                            restart <= 16): about 40 % fewer bytes per Arnoldi
                            step; the stored basis rounds at ~5e-4 relative, so
                            inner_tol should stay >= 1e-3 */
    int augment;         /* PN_SOLVER_IR_GMRES with PN_BASIS_F16: k in [0, 8] corrections
                            of earlier restart cycles (x_i - x_{i-1}, newest first)
                            appended to each cycle's m Krylov directions (LGMRES(m, k));
                            kept across restarts and refinement steps; restart + k
                            <= 16; 0 (default): plain restarted GMRES.  pn_batch_solve
                            ignores it */
} pn_solve_opts;

#define PN_ORTHO_CGS2 0
#define PN_ORTHO_CGS1 1

#define PN_BASIS_F32 0
#define PN_BASIS_F16 1

typedef struct {
    int status;          /* return code of the solve */
    int iterations;      /* inner Krylov iterations (all restarts/outer steps) */
    int outer_iterations;/* IR refinement steps (0 otherwise) */
    double rel_residual; /* final ||Q - A u|| / ||Q|| in FP64 */
    double seconds;      /* host wall time of the call */
    int64_t launches;    /* CUDA kernels the solve launched */
    int precond_applications; /* learned-preconditioner applications */
    int fallback;        /* 1 if the learned preconditioner was dropped for plain GMRES */
} pn_solve_stats;

/* Fill *opts with defaults (CGLS, FP64, tol 1e-6, max_iter 100000, m 60,
 * inner_tol 1e-2, max_outer 50, check_every 10, profile 0, ortho CGS2,
 * precond NULL, basis PN_BASIS_F32). */
void pn_default_solve_opts(pn_solve_opts* opts);

/*
 * Solve A u = Q.  u: device vector in the padded layout, read as the initial
 * guess and overwritten by the solution.  Its element type is PN_F64 for
 * PN_SOLVER_IR_GMRES and opts->precision otherwise.  Reductions accumulate
 * in FP64.  Returns PN_OK, or PN_ERR_NOT_CONVERGED (u holds the last
 * iterate), PN_ERR_BREAKDOWN, PN_ERR_NONFINITE; stats may be NULL.
 * Synchronises the stream.
 */
int pn_solve(pn_handle* h, void* u, const pn_solve_opts* opts, pn_solve_stats* stats, void* stream);

/*
 * Solver workspace of the handle: *bytes (host) = device bytes the solvers
 * hold (Krylov basis, Hessenberg scalars, refinement vectors, LGMRES ring),
 * *allocations = device allocations made for them since pn_create.  A solve
 * allocates only when it needs more workspace than earlier solves on the
 * handle left (the first solve, a larger restart or augmentation); the
 * workspace is kept until pn_destroy, so repeated solves with the same
 * options allocate nothing.  Either output may be NULL.
 */
int pn_get_workspace(const pn_handle* h, int64_t* bytes, int64_t* allocations);

/*
 * Single-scatter source of a collimated beam, as K = (N+1)^2 voxel-centre
 * moments (section "Rendering": the single-scattered light is folded into the
 * emission term, Q = sigma_s int p(w' -> w) L_u(w') dw', with L_u the
 * uncollided light):
 *     Q^{l,m}(x) = sigma_s(x) E(x) g^l Y_{l,m}(w_b),  E = exp(-int sigma_t ds).
 * The beam has unit irradiance, travels along sign * e_axis (axis 0 = x,
 * 1 = y, 2 = z; sign = +1 or -1), enters through the face it points away
 * from, and covers the voxel centres within `radius` of the line through
 * (c0, c1) in the two transverse coordinates (in increasing axis order).
 * The optical depth to a centre is the sum of sigma_t h over the cells before
 * it plus half of its own cell; sigma_t is used as given (no threshold).
 * sigma_t, albedo (or NULL with albedo_const): device arrays R^3 [z][y][x];
 * Q: device output, K x R^3, coefficient k = l*l + l + m major -- the
 * PN_Q_CENTRE_MOMENTS layout of pn_create.  Does not synchronise.
 */
int pn_single_scatter_beam(int N, int R, const void* sigma_t, const void* albedo, double albedo_const, double g,
                           int axis, int sign, double radius, double c0, double c1, void* Q, int dtype, void* stream);

/*
 * out = x interpolated to voxel centres (section "Rendering": the solution is
 * unstaggered before rendering; the extra boundary coefficients are dropped):
 * along each axis on which a coefficient lives on faces, the mean of the two
 * faces of the cell.  x: device vector in the padded layout; out: device
 * array K x R^3, coefficient-major in k = l*l + l + m order, [z][y][x].
 */
int pn_unstagger(pn_handle* h, const void* x, void* out, int dtype, void* stream);

/* ---------------------------------------------------------------------------
 * Learned preconditioner network (an extension; the paper has no network).
 * A 3D convolutional encoder-decoder: four resolution levels of widths
 * widths[0..3] (default 16, 32, 48, 64), two 3x3x3 convolutions with ReLU per
 * encoder level, 2x average pooling down, nearest 2x upsampling up with skip
 * connections by channel concatenation, one 3x3x3 convolution with ReLU per
 * decoder level, and a linear 3x3x3 output layer to c_out channels.  BF16
 * weights and activations on the tensor cores with FP32 accumulation; FP32
 * master weights trained by Adam.  Tensors at the ABI are FP32 device arrays,
 * channels-last [b][z][y][x][c], with Z, Y, X multiples of 8.
 * Host parameter order: per layer (e0a e0b e1a e1b e2a e2b e3a e3b d2 d1 d0
 * out) the weights W[o][c][tap] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1), the
 * convolution reads in[c][p + (dz,dy,dx)]) then the biases b[o].
 */
int pn_cnn_create(pn_cnn** out, int c_in, int c_out, const int widths[4]);
int pn_cnn_destroy(pn_cnn* net);
const char* pn_cnn_last_error(const pn_cnn* net);
int64_t pn_cnn_num_params(const pn_cnn* net);
/* copy parameters (host FP32, count = pn_cnn_num_params) in / out; setting
 * resets the Adam state */
int pn_cnn_set_params(pn_cnn* net, const float* host, int64_t count);
int pn_cnn_get_params(pn_cnn* net, float* host, int64_t count);
/* gradients of the last pn_cnn_backward / pn_cnn_train_step (host FP32) */
int pn_cnn_get_grads(pn_cnn* net, float* host, int64_t count);
/* out = net(in): in [B][Z][Y][X][c_in], out [B][Z][Y][X][c_out] (or NULL) */
int pn_cnn_forward(pn_cnn* net, const float* in, float* out, int B, int Z, int Y, int X, void* stream);
/* parameter gradients of sum(grad_out * net(in)) for the last forward input */
int pn_cnn_backward(pn_cnn* net, const float* grad_out, void* stream);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) with the current gradients */
int pn_cnn_adam_step(pn_cnn* net, double lr, void* stream);
/* forward, loss = mean over samples of |net(in_b) - target_b|^2 / |target_b|^2,
 * backward and one Adam step; *loss_out (host) = the loss before the step
 * (synchronises when loss_out is not NULL).  B <= 4096. */
int pn_cnn_train_step(pn_cnn* net, const float* in, const float* target, int B, int Z, int Y, int X, double lr,
                      double* loss_out, void* stream);

/*
 * Convolution kernel of the network's 3x3x3 layers (forward and input
 * gradient): PN_CNN_CONV_TCGEN05 (default) runs them on the fifth-generation
 * tensor cores (tcgen05.mma, BF16 operands staged by TMA, FP32 accumulators
 * in tensor memory); PN_CNN_CONV_MMA_SYNC on warp-level mma.sync with
 * fragments loaded from global memory (kept for comparison).  Both compute
 * the same products in FP32 accumulation (sums in another order).
 * pn_cnn_take_error: PN_ERR_TIMEOUT (and clears it) if a bounded wait of a
 * tcgen05 convolution ran out since the last call, else PN_OK; synchronises
 * the device.  pn_cnn_train_step (with loss_out) reports the same error.
 */
#define PN_CNN_CONV_MMA_SYNC 0
#define PN_CNN_CONV_TCGEN05  1
int pn_cnn_set_conv_kernel(pn_cnn* net, int kernel);
int pn_cnn_take_error(pn_cnn* net);

/*
 * *out (host) = sum_i x_i y_i for i < n, without allocating anything.
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory where they need a reduction (a host application that
 * owns the whole device-memory budget, a real-time loop that must not take
 * allocator locks or risk running out of memory midway, code that holds
 * device vectors but no pn_handle).  pn_dot needs a handle, whose creation
 * allocates; this call needs none and calls no allocator.
 * x, y: device vectors of n elements of `dtype` (PN_F32 or PN_F64), aligned to
 * their element size; any n in [0, PN_NOALLOC_MAX_ELEMS].  Products and sums
 * are FP64, in a fixed order (deterministic for a given n).
 * Scratch: a fixed 2 MiB __device__ array inside the library (one FP64
 * partial per 8192 elements plus a result slot), held on every device that
 * loads the library until the process exits.  The first call on a device
 * looks up the array's device address (with that device current).  Every
 * call copies the result to the host and synchronises `stream`, so no call
 * can be made on a stream that is being captured into a CUDA graph: such a
 * call returns PN_ERR_ARG before any device work.  All calls share the array
 * and each call overwrites what it uses: calls whose kernels overlap on the
 * GPU (other streams, other host threads) race, so callers must serialise them.
 * Returns PN_OK, PN_ERR_ARG (NULL pointer, bad dtype, misalignment, n < 0,
 * a capturing stream), PN_ERR_TOO_LARGE (n > PN_NOALLOC_MAX_ELEMS) or
 * PN_ERR_CUDA.
 */
#define PN_NOALLOC_MAX_ELEMS (1LL << 31)
int pn_dot_noalloc(const void* x, const void* y, int64_t n, int dtype, double* out, void* stream);

/*
 * The learned preconditioner M(v) = s net(features(v / s)) + P v with
 * s = |v| / sqrt(n), n the number of unknowns (an extension; the paper has
 * no preconditioner).  features(u): for each
 * voxel (x, y, z) < R, channel p = u in plane p at slot (x, y, z), then
 * log(sigma_t h), sigma_s / sigma_t and g (c_in = K + 3); the network's K
 * output channels return to slot (x, y, z) of each plane.  P is the fixed
 * diagonal 1 / (D + 1/h), D the collision-minus-scattering diagonal (the
 * Jacobi inverse where D dominates, h times the identity where transport
 * does).  R must be a multiple of 8.  All vectors are device FP32 in the
 * padded layout of pn_get_layout; network tensors are device FP32
 * channels-last.
 * pn_cnn_features writes scale * features(v) ([R^3][K+3]);
 * pn_cnn_targets writes scale * (e - P r) at the cells' own slots ([R^3][K];
 * r may be NULL: scale * e, the gather of a vector to the network layout);
 * pn_cnn_output writes z = scale * net_out + P v (net_out [R^3][K] scattered
 * to the cells' own slots, or NULL; v may be NULL), the map from network
 * output to a P_N vector used by M and by residual-loss training;
 * pn_cnn_precondition writes z = M(v) (allocates scratch; synchronises).
 */
int pn_cnn_features(pn_handle* h, const float* v, double scale, float* out, void* stream);
int pn_cnn_targets(pn_handle* h, const float* e, const float* r, double scale, float* out, void* stream);
int pn_cnn_output(pn_handle* h, const float* net_out, double scale, const float* v, float* z, void* stream);
int pn_cnn_precondition(pn_handle* h, pn_cnn* net, const float* v, float* z, void* stream);

/*
 * Batched solver: many systems of different grid sizes and orders solved
 * together (an extension; the paper solves one system at a time).  Every
 * phase is one kernel launch over all instances (the operator over
 * (instance, plane, slot chunk) items with each instance's own couplings, the
 * vector kernels over (instance, element chunk) items, persistent grids of a
 * multiple of the SM count); one restart cycle of the inner GMRES(m) (4 m + 5
 * launches, no host synchronisation inside) is captured once as a CUDA graph
 * and replayed; instances converge independently (per-instance flags gate
 * every work item, and an instance that reached its target freezes itself
 * inside the cycle).
 *
 * pn_batch_create: `handles` (count >= 1) are borrowed and must outlive the
 * batch; 3D and 2D handles may be mixed.  restart in [1, 16].  Allocates, per
 * instance, restart + 3 FP32 vectors, one FP64 vector and the FP64 Arnoldi
 * scalars; synchronises `stream`.  Errors: PN_ERR_ARG, PN_ERR_ALLOC,
 * PN_ERR_CUDA.
 * pn_batch_apply: y_i = A_i x_i for every instance in one launch; x, y are
 * host arrays of `count` device pointers (each instance's padded layout,
 * 16-byte aligned, not aliased), dtype PN_F32 or PN_F64.  Stream-ordered on
 * `stream`.
 * pn_batch_solve: solves every A_i u_i = Q_i by FP64 iterative refinement
 * around the batched FP32 GMRES(restart) (opts->solver must be
 * PN_SOLVER_IR_GMRES, opts->restart the batch's restart; tol, inner_tol,
 * max_iter (inner iterations per instance) and max_outer as for pn_solve).
 * u: host array of `count` device pointers to FP64 vectors (initial guesses,
 * overwritten by the solutions); stats: host array of `count` records (status
 * per instance; seconds and launches are the whole batch's).  Synchronises
 * `stream` first and the batch's own stream before returning.  Returns PN_OK
 * when every instance converged, else the first failing instance's status.
 * pn_batch_set_tiling / pn_batch_get_tiling: operator chunk (slots, multiple
 * of 256), vector chunk (elements, multiple of 1024) and CTAs per SM of the
 * two kinds of persistent grid.
 * pn_batch_tune: the autotuner: times the batched operator over operator
 * chunk {4096, 16384, 65536} x {2, 4, 8} CTAs per SM, the per-instance tiled
 * operator path against the best of those, and the Arnoldi vector kernels
 * over vector chunk {16384, 65536, 262144} x {2, 4, 8}, on this batch, and
 * keeps the fastest of each (pn_batch_get_tiling, pn_batch_get_op_path).  It
 * times the instances the batched launches take under the current solo
 * threshold (pn_batch_set_solo), so call it after changing that threshold.
 * pn_batch_set_mode: PN_BATCH_GRAPH (default) replays the captured cycle;
 * PN_BATCH_PERSISTENT runs each cycle as ONE cooperative launch (a grid of
 * resident CTAs, two per SM) whose phases are separated by grid barriers.
 * Every barrier wait is bounded by spin_limit polls of about 100 ns; when one
 * runs out the kernel ends and pn_batch_solve returns PN_ERR_TIMEOUT (the
 * iterates are then those of the last completed cycle plus a partial one).
 * pn_batch_barrier_test: one cooperative launch of `blocks` CTAs (at most the
 * resident count) running a single barrier that expects `expected` >= blocks
 * arrivals with the given spin limit: PN_OK and *timed_out = 0 when it
 * completes (expected == blocks), PN_ERR_TIMEOUT and *timed_out = 1 when the
 * wait runs out (expected > blocks), for tests of the timeout path.
 */
#define PN_BATCH_GRAPH      0
#define PN_BATCH_PERSISTENT 1
typedef struct pn_batch pn_batch;
int pn_batch_create(pn_batch** out, pn_handle* const* handles, int count, int restart, void* stream);
int pn_batch_destroy(pn_batch* batch);
const char* pn_batch_last_error(const pn_batch* batch);
int pn_batch_apply(pn_batch* batch, const void* const* x, void* const* y, int dtype, void* stream);
int pn_batch_solve(pn_batch* batch, double* const* u, const pn_solve_opts* opts, pn_solve_stats* stats,
                   void* stream);
int pn_batch_set_tiling(pn_batch* batch, int64_t op_chunk, int64_t vec_chunk, int op_ctas_per_sm,
                        int vec_ctas_per_sm);
int pn_batch_get_tiling(const pn_batch* batch, int64_t* op_chunk, int64_t* vec_chunk, int* op_ctas_per_sm,
                        int* vec_ctas_per_sm);
int pn_batch_tune(pn_batch* batch, void* stream);
int pn_batch_set_mode(pn_batch* batch, int mode, long long spin_limit);
/* Instances with at least min_unknowns unknowns fill the GPU alone and gain
 * nothing from sharing launches: pn_batch_solve solves them first with
 * pn_solve (the same FP64 refinement around FP32 GMRES with one Gram-Schmidt
 * pass and the batch's restart), three at a time from three host threads on
 * three of the batch's streams, largest first (each solve's result is that
 * of a solve on its own), and the rest together in the batched launches, whose work lists then hold no chunk of a solo instance
 * (pn_batch_apply restores the full lists).  Default 2^18; min_unknowns <= 0
 * batches every instance. */
int pn_batch_set_solo(pn_batch* batch, long long min_unknowns);
int pn_batch_barrier_test(int blocks, int expected, long long spin_limit, int* timed_out, void* stream);
/* Arnoldi-step operator of the graph mode: 1 = every 3D instance the tiled
 * FP32 kernel serves gets its own gated launch on one of eight side streams
 * (independent branches of the captured graph, run concurrently; the rest
 * share one generic launch), 0 = one generic launch over all instances.
 * Default 1; pn_batch_tune keeps the faster.  The persistent mode always uses
 * the generic launch (a cooperative kernel cannot launch others). */
int pn_batch_set_op_path(pn_batch* batch, int tiled);
int pn_batch_get_op_path(const pn_batch* batch, int* tiled);

/*
 * Tile plan of the FP32 operator (3D handles): the z-marching tiled kernel
 * splits each (x, y) tile column into z chunks so that about ctas_per_sm CTAs
 * per SM are launched (default 4; larger values shorten the chunks).
 * pn_tune_apply times the FP32 apply for ctas_per_sm in {1, 2, 4, 8}, each main
 * kernel (below) and both schedules of the face-column kernel (the outputs
 * right of the tiles: concurrently on a side stream, or after the main kernel)
 * on this handle (allocates two scratch vectors; synchronises `stream`), keeps
 * the fastest and reports its ctas_per_sm and time per apply (either output
 * may be NULL).  While programmatic dependent launch is enabled (pn_set_pdl,
 * the default) each timing is a chain of four applies launched as the
 * solvers launch them (face-column kernel first, the main kernel overlapping
 * it), so the plan is chosen for the solvers' Arnoldi steps; pn_get_apply_plan reports the whole plan (any output may be NULL);
 * pn_set_apply_tiling sets ctas_per_sm directly (1..16).  Results do not
 * depend on the plan except for the order of the residual's partial sums.
 */
int pn_tune_apply(pn_handle* h, void* stream, int* ctas_per_sm, double* best_ms);
int pn_set_apply_tiling(pn_handle* h, int ctas_per_sm);
int pn_get_apply_plan(const pn_handle* h, int* ctas_per_sm, int* kernel, int* face_serial);

/*
 * Main kernel of the tiled FP32 operator (3D handles with the vacuum
 * boundary), both over 32 x 4 column tiles marching in z:
 *   PN_APPLY_KERNEL_TMA (default): each parity class's input planes are
 *     staged in shared memory by TMA tensor copies (one 4D box per class and
 *     z-slice; inactive slots arrive as 0), and the four thread groups of a
 *     CTA compute equal shares of the rows.  Its mbarrier waits are bounded
 *     (about 2 s); one that runs out makes the next pn_solve return
 *     PN_ERR_TIMEOUT.
 *   PN_APPLY_KERNEL_REGISTER: each thread loads its columns' values of two
 *     z-adjacent classes into registers and stages them in shared memory.
 * Both give bitwise-identical outputs (the residual norm's partial sums of
 * r^2 are formed over other sets of outputs, so it agrees to their FP32
 * rounding).  pn_tune_apply times both (with every z
 * chunking) and keeps the fastest.  pn_set_apply_kernel returns
 * PN_ERR_UNSUPPORTED if the TMA kernel cannot serve the handle (no driver
 * entry point for tensor maps); handles the tiled operator does not serve
 * ignore the setting.  pn_get_apply_kernel reports the kernel that runs.
 */
#define PN_APPLY_KERNEL_REGISTER 0
#define PN_APPLY_KERNEL_TMA      1
int pn_set_apply_kernel(pn_handle* h, int kernel);
int pn_get_apply_kernel(const pn_handle* h, int* kernel);

/*
 * L2 residency of the FP16-basis GMRES (PN_BASIS_F16): while it runs, its two
 * FP32 step vectors (A v and the newest basis vector, each written and read
 * again within every Arnoldi step) are kept in L2 by a persisting
 * access-policy window on the solver's stream, up to the device's persisting
 * capacity, when the two fit in L2 (larger ones are left alone); afterwards the window is closed, the persisting lines released and
 * the context's persisting-lines limit restored.  pn_solve runs on a stream of
 * its own, ordered after `stream` on entry and before it on exit.  on = 1
 * (default) or 0.  Results do not depend on it.
 */
int pn_set_l2_residency(pn_handle* h, int on);

/*
 * Vector kernels of the FP16-basis GMRES: bit 0 of `mask` stages the fused
 * CGS1 step's streams (w and the basis vectors), bit 1 the multi-axpy's, in
 * shared memory by bulk copies (TMA, 1024-element chunks, every G-th chunk
 * to each of G blocks, two slots per block, three blocks per SM) for steps
 * with at least five basis vectors (with fewer the direct form is faster); a
 * clear bit loads them directly.
 * Default 3.  Both forms compute the same products; the multi-dot's sums are
 * formed in another order, so results agree to rounding.
 */
int pn_set_stream_kernels(pn_handle* h, int mask);

/*
 * Self-test of the bounded mbarrier wait that the TMA-staged kernels use
 * (an aid for tests; the paper has no counterpart).  One CTA arms an
 * mbarrier: with deliver = 1 the phase completes at once; with deliver = 0 it
 * expects 16 bytes that no copy brings, so the wait runs out after limit_ns
 * (1 ns .. 10 s) of the GPU's global timer, sets the fault word and returns.
 * No copy is issued.  With a handle the fault word is the handle's own (the
 * one the operator and vector kernels set), so the next pn_solve on h returns
 * PN_ERR_TIMEOUT and clears it; with h == NULL a temporary word is used.
 * *timed_out (host) = 1 when this launch's wait ran out (a word already set
 * before the call reads 0).  Returns PN_ERR_TIMEOUT when it did, PN_OK when
 * the phase completed; PN_ERR_ARG, PN_ERR_ALLOC, PN_ERR_CUDA otherwise.
 * Synchronises `stream`.
 */
int pn_wait_timeout_test(pn_handle* h, int deliver, long long limit_ns, int* timed_out, void* stream);

/*
 * Programmatic dependent launch in the FP16-basis GMRES (PN_BASIS_F16): the
 * kernels of each Arnoldi step (operator, fused CGS1 step, multi-axpy) are
 * launched so that each may start while the one before it finishes; each
 * kernel waits for its predecessor's results before it reads them (copies of
 * inputs that are already complete go out before the wait).  on = 1
 * (default) or 0.  Results do not depend on it (bitwise).
 */
int pn_set_pdl(pn_handle* h, int on);

/*
 * Arithmetic peak of the current GPU (a measurement aid; the paper has no
 * counterpart): *gflops_out (host) = FMA throughput in GFLOP/s (2 flops per
 * FMA) of a kernel of independent FP64 (dtype PN_F64) or FP32 (PN_F32) FMA
 * chains filling every SM, best of five timed launches.  The denominator of
 * the roofline of kernels bound by FP64 arithmetic.  Allocates 8 bytes and
 * two events; synchronises `stream`.
 */
int pn_fma_peak(int dtype, double* gflops_out, void* stream);

/*
 * Bandwidth of the tiled operator's memory access pattern without its
 * arithmetic (a measurement aid; the paper has no counterpart): a copy of
 * `planes` (4..64, a multiple of 4) coefficient planes of an R^3 grid (R in
 * [128, 512], a multiple of tile_x) in the library's plane-major padded
 * layout, by CTAs of 512 threads that march tiles of tile_x x (128 / tile_x)
 * columns (tile_x in {32, 64, 128}) through z, each thread holding `slices`
 * (1, 2 or 4) z-slices x planes / 4 loads in flight: with 64 planes, 32, 64
 * or 128 KB in flight per CTA.  *gbs_out (host) = 2 x 4 x planes x R (R+1)^2
 * bytes / the best of five timed copies, in GB/s.  Allocates two buffers of
 * about planes x 4 (R+1)^3 bytes (PN_ERR_ALLOC if they do not fit) and two
 * events; synchronises `stream`.  PN_ERR_ARG for arguments out of range.
 */
int pn_access_probe(int R, int planes, int tile_x, int slices, double* gbs_out, void* stream);

/* Kernel classes reported by pn_profile_get. */
#define PN_PROF_APPLY    0   /* pn_apply / pn_apply_t operator launches */
#define PN_PROF_RESIDUAL 1   /* residual operator launches */
#define PN_PROF_MDOT     2   /* multi-vector inner products (GMRES) */
#define PN_PROF_MAXPY    3   /* multi-vector updates (GMRES) */
#define PN_PROF_DOT      4   /* single inner products and their reductions */
#define PN_PROF_VECTOR   5   /* axpy-type updates, scaling, conversions */
#define PN_PROF_SCALAR   6   /* one-thread scalar kernels and final reductions */
#define PN_PROF_PRECOND  7   /* learned-preconditioner applications (network + glue) */
#define PN_PROF_KINDS    8

/*
 * Per-class totals of the last pn_solve run with opts->profile = 1 (zeros
 * otherwise): summed event-timed milliseconds, number of launches, and the
 * algorithmic bytes those launches move (every active unknown read or
 * written once per vector operand, parameter fields once).  Host pointers;
 * any may be NULL.  No synchronisation (the solve already synchronised).
 */
int pn_profile_get(const pn_handle* h, int kind, double* ms, int64_t* launches, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* PN_GB300_H */
