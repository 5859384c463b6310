/*
 * mera.h -- C ABI of libmera: energy/gradient and Riemannian optimisation of
 * a scale-invariant binary (default) or ternary MERA, or of a uniform MPS, on
 * one GB300 (sm_103a).
 *
 * Method: Hauru, Van Damme, Haegeman, "Riemannian optimization of isometric
 * tensor networks" (arXiv:2007.03638).  Section numbers and equation labels
 * below refer to that paper.
 *
 * Object model
 * ------------
 * A mera_t owns every piece of device state of one optimisation problem: the
 * tensors (the current point), the Hamiltonian, the ascended operators and
 * density matrices, the Krylov warm starts of the scale-invariant layer, the
 * last gradient, the preconditioner's density matrices and the L-BFGS/CG
 * history.  All work is issued on the CUDA stream given to mera_create.
 *
 * Tensor list
 * -----------
 * The point is the list [u_0, w_0, u_1, w_1, ..., u_L, w_L] (2*(n_trans+1)
 * matrices): n_trans transition layers followed by the scale-invariant
 * layer L.  With layer dimensions chi_0 = d_b, chi_{l+1} = min(chi, chi_l^2)
 * (and chi_L = chi):
 *   u_l : (chi_l^2) x (chi_l^2) unitary, row-major, u[f_a f_b, x_a x_b]
 *         (rows: the fine pair it outputs; columns: the pair of isometry
 *         outputs it acts on; left leg most significant);
 *   w_l : (chi_l^2) x (chi_{l+1}) isometry, row-major, w[x_a x_b, k],
 *         w^dag w = 1 (w_L is chi^2 x chi).
 * (The ternary network, mera_config.network = MERA_TERNARY, has
 * chi_{l+1} = min(chi, chi_l^3) and w_l of (chi_l^3) x (chi_{l+1}); see
 * mera_network.)
 * Tangent vectors, partial derivatives and gradients use the same shapes.
 * mera_tensor_shape() reports them.  Element type: double (MERA_F64) or
 * interleaved complex double (MERA_C128: real part first, the layout of C99
 * double _Complex).  In a mixed-precision mode every complex contraction
 * of the MERA networks runs as four real tensor-core products of the real
 * and imaginary parts (Re C = Re A Re B - Im A Im B, Im C = Re A Im B +
 * Im A Re B; conjugated operands by sign), the rest in FP64 as for real
 * data (the MPS serves FP64 only, see MERA_MPS).  For
 * complex data the inner product of the tangent space is Re Tr(X^dag Y) and
 * the projections, retractions and preconditioner use conjugate transposes
 * where the real case has transposes (Sec. 2.3, Sec. 3).
 *
 * Pointers
 * --------
 * Every data pointer argument may be host or device memory (unified virtual
 * addressing decides); the library copies in or out on its stream and the
 * caller keeps ownership.  Calls return after the stream work they need for
 * their scalar outputs has completed; array outputs are complete when the
 * call returns.
 *
 * Errors
 * ------
 * Every int-returning call returns MERA_OK (0) or a negative MERA_ERR_* code;
 * mera_strerror() names it and mera_last_error() gives the detail of the last
 * failure on that object.  No call aborts or exits; after an error the object
 * stays valid (the point is unchanged unless stated otherwise).
 */
#ifndef MERA_H
#define MERA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mera_ctx* mera_t;

enum {
    MERA_OK = 0,
    MERA_ERR_ARG = -1,            /* invalid argument / shape / config        */
    MERA_ERR_OOM = -2,            /* device allocation failed                 */
    MERA_ERR_NONFINITE = -3,      /* NaN/Inf in an input, energy or gradient  */
    MERA_ERR_NOCONV = -4,         /* Krylov solve or line search not converged*/
    MERA_ERR_DEVICE_TIMEOUT = -5, /* a bounded device-side wait expired       */
    MERA_ERR_NOT_ISOMETRIC = -6,  /* input tensor violates W^dag W = 1        */
    MERA_ERR_CUDA = -7,           /* CUDA runtime error                       */
    MERA_ERR_UNSUPPORTED = -8     /* valid request the library does not serve */
};

typedef enum { MERA_F64 = 0, MERA_C128 = 1 } mera_dtype;

/* Arithmetic of the bulk contractions (ascending/descending maps and
 * environments).  FP64 keeps everything in double; the mixed modes run the
 * contractions on tensor cores with FP32 accumulation and keep the Krylov
 * solves, reductions, geometry and line search in FP64.  Each operand x is
 * split into a high and a low plane, x = hi + lo, and a product takes
 * hi*hi + hi*lo + lo*hi:
 *   MERA_PREC_3XTF32      TF32 planes (about 22 significant bits), kind::tf32;
 *   MERA_PREC_SPLIT_BF16  BF16 planes (about 16 bits), kind::f16 at twice the
 *                         TF32 rate;
 *   MERA_PREC_SPLIT_FP16  FP16 planes of the operand scaled by a power of two
 *                         chosen from its largest entry (about 22 bits, as
 *                         3xTF32, at the BF16 rate); the scale is divided out
 *                         exactly when the product is stored. */
typedef enum { MERA_PREC_FP64 = 0, MERA_PREC_3XTF32 = 1, MERA_PREC_SPLIT_BF16 = 2,
               MERA_PREC_SPLIT_FP16 = 3 } mera_prec;

typedef struct {
    int d_b;           /* bottom site dimension (4: two spins blocked)        */
    int chi;           /* bond dimension of the scale-invariant layer          */
    int n_trans;       /* number of transition layers (>= 1; 0 for an MPS)    */
    int dtype;         /* mera_dtype                                           */
    int prec;          /* mera_prec                                            */
    int w_stiefel;     /* 0: isometries on the Grassmann manifold (Sec. 4),
                          1: treat them as Stiefel points                      */
    int precond;       /* 1: Hilbert-space preconditioner (Sec. 3, Sec. 4)     */
    int krylov_dim;    /* restart length of the scale-invariant Krylov solves  */
    int krylov_maxiter;/* max matrix-vector products per Krylov solve          */
    double krylov_tol; /* relative residual target of the Krylov solves        */
    int recompute_env; /* 1: recompute each transition layer's ascending
                          intermediates in the gradient pass and keep one set
                          of them for all layers and both sides (binary
                          network; at chi = 32 in a mixed mode about 41 GB
                          less); 0: reuse the ones the up-sweep keeps per
                          layer and side                                       */
    int lbfgs_m;       /* L-BFGS memory length                                 */
    int b_chunk;       /* slice length of the middle coarse leg in the chi^9
                          contraction chain (must divide the coarse bond
                          dimension; 0 = automatic: no slicing while the
                          7-leg intermediate has at most 2^30 entries)        */
    int network;       /* mera_network: MERA_BINARY (default), MERA_TERNARY
                          or MERA_MPS                                          */
    int z2;            /* 1: Z2-symmetric problem: every leg is graded (the
                          first half of its basis even, the rest odd), the
                          Hamiltonian term and the tensors must be symmetric
                          (an entry between index tuples of different total
                          charge is zero, Sec. 6; mera_create /
                          mera_set_tensors return MERA_ERR_ARG when one
                          exceeds 1e-12 of the largest entry), and every
                          contraction of the networks runs as its two charge
                          sectors, a quarter of the dense work; the results
                          are those of the dense path.  Ternary network; the
                          binary one where its chi^9 chain needs no slicing
                          (chi_l^6 chi_{l+1} <= 2^30 on every layer, chi <= 16
                          from d_b = 4: blocked spin pairs must then be in a
                          basis whose first half is even); otherwise, and for
                          an MPS, MERA_ERR_UNSUPPORTED.                      */
    double device_wait_s; /* limit, in seconds, of every wait of the
                          tensor-core contraction kernel's pipeline (0 <
                          device_wait_s <= 60; default 1): a wait that
                          expires ends the kernel early and the call returns
                          MERA_ERR_DEVICE_TIMEOUT (see mera_set_device_wait) */
} mera_config;

/* Network of the MERA (Sec. 4).  MERA_BINARY: the binary MERA described
 * above, three-site operators.  MERA_TERNARY: the ternary MERA of the
 * paper's benchmark: w_l is (chi_l^3) x (chi_{l+1}) (w[x_a x_b x_c, k], the
 * coarse site to a fine triple), u_l is (chi_l^2) x (chi_l^2) on the pairs
 * that straddle two triples, chi_{l+1} = min(chi, chi_l^3), and operators
 * (h3 of mera_create, the level operators) are two-site: (d_b^2) x (d_b^2)
 * terms whose translates sum to H, energy per site.  For the ternary
 * network the preconditioner's rho_w is the one-site marginal of the level
 * density matrix and rho_u the state on the two isometry outputs a u acts
 * on; every entry point serves both networks. */
typedef enum { MERA_BINARY = 0, MERA_TERNARY = 1, MERA_MPS = 2 } mera_network;

/* MERA_MPS: the uniform (one-site translation-invariant) infinite MPS of
 * Sec. 5 on the same geometry and optimisers.  Config: d_b = physical
 * dimension d, chi = bond dimension D (>= 1), n_trans = 0, prec =
 * MERA_PREC_FP64, w_stiefel = 0 (b_chunk and recompute_env are unused).
 * The point is one tensor A, (D d) x D row-major, A[a s, b] (rows: left
 * virtual leg then physical leg; column: right virtual leg), left-canonical:
 * A^dag A = 1 (Eq. mps_isometricity), a point of the Grassmann manifold
 * (right unitary rotations are gauge).  h3 of mera_create is a two-site
 * term, (d^2) x (d^2), h[s t, s' t'] (rows the bra pair); the cost is the
 * energy per site of the normalised state, e = Tr(T_h(rho)) with rho the
 * unit-trace fixed point of E_R(y) = sum_s A^s y A^s^dag
 * (Eq. mps_right_transfermatrix).  mera_energy_grad gives the partial
 * derivative of Eq. mps_derivative (D = 2 de/d conj(A); the left and right
 * energy environments solve (1 - E_L + |1)(rho|) H_l = h_l and
 * (1 - E_R + |rho)(1|) H_r = h_r by GMRES, h_l and h_r being the
 * left- and right-contracted term h - e 1) and its Grassmann projection;
 * the preconditioner is X -> X (rho + delta 1)^(-1), delta = |G|^2
 * (Eq. mps_preconditioning with the regularisation of Sec. 5).  Other
 * configurations return MERA_ERR_ARG (shape) or MERA_ERR_UNSUPPORTED
 * (mixed precision, Stiefel); mera_ev_sweep and the server return
 * MERA_ERR_UNSUPPORTED for an MPS. */

/* Fill *cfg with defaults for (d_b, chi, n_trans): binary network, F64,
 * FP64 contractions, Grassmann isometries, preconditioner on, Krylov dim 20,
 * 2000 products, tol 1e-14, no recomputation, m = 8, device waits of 1 s. */
void mera_config_default(mera_config* cfg, int d_b, int chi, int n_trans);

/* Create a problem.  h3 is the 3-site Hamiltonian term on bottom sites,
 * a (d_b^3) x (d_b^3) row-major matrix h[f0 f1 f2, g0 g1 g2] of the config's
 * element type whose translates sum to H (the cost is the energy per bottom
 * site, C = Tr(h rho), Sec. 4); for the ternary network and the MPS a
 * two-site term, (d_b^2) x (d_b^2).  stream: a cudaStream_t (NULL = default
 * stream).  The tensors start as the identity-disentangler / first-columns
 * isometry point until mera_set_tensors or mera_init_random is called.
 * MERA_ERR_ARG (before any device work) for a config outside its ranges:
 * unknown dtype, prec or network; w_stiefel, precond, recompute_env or z2
 * not 0 or 1; krylov_tol not in (0, 1); krylov_maxiter, krylov_dim or lbfgs_m
 * below 1; a negative b_chunk; device_wait_s not in (0, 60]; a Hamiltonian
 * term that is not Hermitian (|h - h^dag| above 1e-10 of its largest
 * entry).  MERA_ERR_NONFINITE for a Hamiltonian term with a NaN or an
 * infinite entry. */
int mera_create(const mera_config* cfg, const void* h3, void* stream, mera_t* out);
int mera_destroy(mera_t m);

/* Number of tensors (2*(n_trans+1); 1 for an MPS) and the shape of tensor i. */
int mera_num_tensors(mera_t m);
int mera_tensor_shape(mera_t m, int i, int64_t* rows, int64_t* cols);

/* Copy the point in / out (arrays in the tensor-list order above).
 * mera_set_tensors checks that every entry is finite (MERA_ERR_NONFINITE)
 * and W^dag W = 1 to 1e-10 (MERA_ERR_NOT_ISOMETRIC), and clears the
 * optimiser history; on an error the point is unchanged. */
int mera_set_tensors(mera_t m, const void* const* tensors);
int mera_get_tensors(mera_t m, void* const* tensors);

/* Fill the point with seeded random isometries: the sign-fixed
 * QR-of-Gaussian initialisation (the thin QR factor of a Gaussian matrix,
 * R's diagonal real and positive), tensor by tensor in the order of the
 * tensor list.  The Gaussian matrix of tensor i is row-major (interleaved
 * real and imaginary parts, each N(0,1), for MERA_C128), and its entries are
 * g_0, g_1, ... of stream i: with SplitMix64 (Steele, Lea, Flood, OOPSLA
 * 2014) written x_k(s) = mix(s + k * 0x9E3779B97F4A7C15) for k >= 1 and
 * mix(z) = z3 of z1 = (z ^ z >> 30) * 0xBF58476D1CE4E5B9,
 * z2 = (z1 ^ z1 >> 27) * 0x94D049BB133111EB, z3 = z2 ^ z2 >> 31 (64-bit),
 * base_i = x_{i+1}(seed), u_k = ((x_k(base_i) >> 11) + 0.5) * 2^-53, and for
 * every pair j = 0, 2, 4, ...: r = sqrt(-2 ln u_{j+1}),
 * t = 2 pi u_{j+2}, g_j = r cos t, g_{j+1} = r sin t (Box-Muller).  With
 * z2 = 1 each charge block (rows and columns of charge q in ascending order)
 * is factored on its own and the entries between charges are zero.  Host
 * computation (once per problem), then a copy to the device; resets the
 * optimiser history like mera_set_tensors.  MERA_ERR_ARG if a charge block
 * has fewer rows than columns. */
int mera_init_random(mera_t m, uint64_t seed);

/* Energy per bottom site C = Tr(h rho) and the Riemannian gradient G at the
 * current point (Sec. 4 with App. B; G_v is the tangent projection of the
 * partial derivative D_v = 2 dC/d conj(v), Eqs. stiefel_gradient /
 * grassmann_gradient).  grad may be NULL; otherwise grad[i] receives G_i.
 * D (unprojected) is written to deriv[i] if deriv is not NULL.  Also
 * refreshes the density matrices used by mera_precondition. */
int mera_energy_grad(mera_t m, double* energy, void* const* grad, void* const* deriv);

/* Energy per bottom site only (ascending maps, scale-invariant fixed point,
 * Tr(h_L rho_S); Sec. 4, App. B): no environment series, no reverse pass. */
int mera_energy(mera_t m, double* energy);

/* G = projection of arbitrary D onto the tangent space at the current point. */
int mera_project(mera_t m, const void* const* D, void* const* G);

/* g(X, Y) = sum_v Re Tr(X_v^dag Y_v)  (Euclidean metric, Sec. 2.2). */
int mera_inner(mera_t m, const void* const* X, const void* const* Y, double* out);

/* Vector transport along the retraction from the current point (Eq. transport):
 * Y_i <- exp(alpha Q_{X_i}) Y_i, in place.  Call before mera_retract moves the
 * point.  MERA_ERR_NONFINITE if X has a NaN or infinite entry. */
int mera_transport(mera_t m, const void* const* X, double alpha, void* const* Y);

/* Move the current point along the exponential retraction (Eq. retraction):
 * W_i <- exp(alpha Q_{X_i}) W_i, followed by re-isometrisation (polar factor).
 * If Xprime is not NULL it receives dR/dalpha = exp(alpha Q_X) X.
 * MERA_ERR_NONFINITE (point unchanged) if X has a NaN or infinite entry. */
int mera_retract(mera_t m, const void* const* X, double alpha, void* const* Xprime);

/* Hilbert-space preconditioner (Eq. preconditioner_solution) with the
 * density matrices of the last mera_energy_grad and delta_v = |G_v|. */
int mera_precondition(mera_t m, const void* const* X, void* const* Xt);

typedef struct {
    int iter;           /* iterations done so far                       */
    double energy;      /* energy per bottom site after the step         */
    double gnorm;       /* |G| after the step                            */
    double alpha;       /* accepted step                                 */
    int n_evals;        /* energy_grad evaluations in this step          */
    int ls_ok;          /* 1: Wolfe / approximate Wolfe met              */
    int krylov_matvecs; /* superoperator applications in this step       */
} mera_iter_info;

/* One full Riemannian L-BFGS iteration (Sec. 3): two-loop direction with the
 * preconditioned initial Hessian, Hager-Zhang line search along the
 * retraction, transport of the history.  The first call evaluates the
 * gradient at the current point. */
int mera_lbfgs_step(mera_t m, mera_iter_info* info);

/* One nonlinear conjugate-gradient iteration (Hager-Zhang beta, Sec. 3). */
int mera_cg_step(mera_t m, mera_iter_info* info);

/* One Riemannian gradient-descent iteration (Sec. 3): retraction along the
 * negative preconditioned gradient, the Hager-Zhang step started at the
 * previous accepted step.  Clears the L-BFGS/CG history. */
int mera_gd_step(mera_t m, mera_iter_info* info);

/* One Evenbly-Vidal sweep, the comparator of the paper's optimisers (Sec. 4
 * and App. ev_steplimit): for every tensor in the order u_0, w_0, ..., u_S,
 * w_S, the environment D of the cost with the shifted term
 * h3 - gamma 1 is computed at the current point (one full evaluation) and the
 * tensor is replaced by -Q, Q the isometric polar factor of D = Q P (the sign
 * leaves the state and its energy unchanged; -Q keeps the tensor's sign near a
 * fixed point).  gamma should make h3 - gamma 1 negative definite (its largest
 * eigenvalue plus a margin); it acts as an inverse step size.  Clears the
 * L-BFGS/CG history.  info: energy (unshifted) and |G| at the new point from
 * one more evaluation, n_evals = number of tensors + 1, alpha = 0.
 * MERA_ERR_ARG for a non-finite gamma; MERA_ERR_UNSUPPORTED for an MPS. */
int mera_ev_sweep(mera_t m, double gamma, mera_iter_info* info);

typedef struct {
    int method;       /* 0 = L-BFGS, 1 = CG, 2 = gradient descent */
    int maxiter;
    double gtol;      /* stop when |G| < gtol                 */
} mera_solve_opts;

typedef struct {
    int iters;
    int n_evals;
    double energy;
    double gnorm;
    int converged;
} mera_solve_result;

/* Run iterations until |G| < gtol or maxiter. */
int mera_solve(mera_t m, const mera_solve_opts* opts, mera_solve_result* res);

/* Device bytes a problem with this config holds (for admission control). */
size_t mera_footprint_bytes(const mera_config* cfg);

/* Number of kernel launches issued by this object so far. */
int64_t mera_launch_count(mera_t m);

/* Counters of one object since its creation (or the last reset).  The
 * contraction kernel's device time is summed only over launches issued while
 * profiling is on (a CUDA event pair on the object's stream around each
 * launch); reading synchronises the stream. */
typedef struct {
    int64_t launches;          /* all kernels                                   */
    int64_t gett_launches;     /* tensor-contraction kernel launches            */
    double gett_flops;         /* algorithmic flops of those launches (2 M N K) */
    int64_t gett_timed;        /* contraction launches timed with events        */
    double gett_ms;            /* their summed device time                      */
    int64_t energy_grad_calls; /* energy/gradient evaluations                    */
    int64_t krylov_matvecs;    /* scale-invariant superoperator applications    */
} mera_stats;
int mera_get_stats(mera_t m, mera_stats* out, int reset);
int mera_profile(mera_t m, int enable);
/* Write the per-shape table of the contractions timed while profiling was on
 * (since creation or the last reset of mera_get_stats) to the file `path` as
 * CSV lines "M,N,K,path,calls,ms,tflops": path 0 is the FP64 contraction
 * kernel, otherwise 1000 * (1 + tensor-core kind: 0 TF32, 1 BF16) + 100 *
 * epilogue store mode;
 * tflops counts 2 M N K per call.  Rows with K = 0 time other phases:
 * path 91xx / 92xx the packing of a tensor-core product's first / second
 * operand into split planes (M, N = rows, packed length; xx = 10 if the
 * source's stride-1 leg is a row leg, + 1 if the source is float), path
 * 9300 one eigendecomposition of the preconditioner (M = N = order).
 * Synchronises the object's stream.
 * MERA_ERR_ARG if the file cannot be written. */
int mera_profile_dump(mera_t m, const char* path);

/* ---------------------------------------------------------------- serving --
 * Many optimisations on one GPU (no counterpart in the paper; the request
 * stream of the serving workload).  Requests are queued in arrival order and
 * admitted while their device footprint (mera_footprint_bytes) fits in the
 * memory budget; each admitted request owns a mera_t on its own stream, so
 * its state stays on the device until it finishes, and n_workers host
 * threads take turns stepping the running requests one iteration at a time
 * (their kernels overlap on the GPU).  Requests with the same configuration
 * of the binary network (real tensors, unsliced chi^9 chain: chi <= 16 from
 * d_b = 4) form a cohort: their energy/gradient evaluations that are due at
 * the same time (within a gathering window of 1.5 ms) run together, every
 * contraction one batched launch over up to 8 of them and their Krylov
 * solves in lockstep, on the cohort's own stream; the cohort's workspace
 * (the planes of 8 members) counts against the budget while it lives.  A
 * request stops when |G| < gtol or after maxiter iterations.  Results do not
 * depend on the mix: each request's arithmetic is that of the request
 * alone. */
typedef struct mera_server* mera_server_t;

typedef struct {
    int state;        /* 0 queued, 1 running, 2 done, 3 failed                 */
    int error;        /* MERA_ERR_* of a failed request                         */
    int iters;        /* iterations done                                         */
    int n_evals;      /* energy/gradient evaluations                             */
    double energy;    /* energy per bottom site after the last iteration         */
    double gnorm;     /* |G| after the last iteration                            */
    double t_submit;  /* seconds since the server started                        */
    double t_admit;   /* -1 until admitted                                       */
    double t_done;    /* -1 until finished                                       */
    size_t bytes;     /* device footprint the request was admitted with          */
    char message[160];/* detail of a failure (mera_last_error of the request)    */
    int deferred;     /* times its creation ran out of device memory while other
                         requests ran, so that it went back to the head of the
                         queue until one of them finished (a creation that runs
                         out of memory with nothing else running fails)       */
    int batched_evals;/* energy/gradient evaluations that ran together with
                         other requests of its cohort (batched launches)       */
} mera_request_status;

int mera_server_create(size_t mem_budget_bytes, int n_workers, mera_server_t* out);
/* Copies cfg, h3 and the starting tensors (host pointers) into the queue.
 * method: 0 L-BFGS, 1 CG.  MERA_ERR_OOM if the request alone exceeds the budget. */
int mera_server_submit(mera_server_t sv, const mera_config* cfg, const void* h3, const void* const* tensors,
                       int method, double gtol, int maxiter, int64_t* id);
int mera_server_poll(mera_server_t sv, int64_t id, mera_request_status* st);
/* Wait until every submitted request has finished (MERA_ERR_NOCONV on timeout). */
int mera_server_wait(mera_server_t sv, double timeout_s);
/* Stop the workers after their current step; unfinished requests are dropped. */
int mera_server_destroy(mera_server_t sv);

/* C = A B for row-major double matrices A (M x K), B (K x N), C (M x N) on
 * the device, with the contraction arithmetic of the given mera_prec:
 * FP64 (the FP64 contraction kernel) or the tensor-core kernel with 3xTF32,
 * split-BF16 or scaled split-FP16 operands and FP32 accumulation.  Exposes the arithmetic of each
 * mode for checking (Sec. 4 contractions are built from this product);
 * allocates its temporary operand planes.  MERA_ERR_DEVICE_TIMEOUT if a
 * bounded device-side wait expired. */
int mera_gemm(int prec, int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C,
              void* stream);

/* Forget the Krylov warm starts: the next evaluation starts its
 * scale-invariant solves (App. B) from the default guesses (rho = 1/chi^3,
 * x = h_S) instead of the last solutions.  Evaluations from a fresh object,
 * or after this call, at the same point are bit-identical (every reduction
 * runs in a fixed order); warm-started ones agree to the Krylov tolerance.
 * The paper has no counterpart of this entry point. */
int mera_reset_warm_starts(mera_t m);

/* Change the limit of the tensor-core kernel's pipeline waits of an
 * existing object (mera_config.device_wait_s; 0 < seconds <= 60, else
 * MERA_ERR_ARG).  When a wait expires the kernel stops issuing work, waits
 * for the copies and tensor-core operations it has already issued, frees its
 * tensor memory and returns; the call that ran it returns
 * MERA_ERR_DEVICE_TIMEOUT and the object stays usable: its point is
 * unchanged and the next evaluation starts its Krylov solves afresh.  A
 * limit far below the kernel's normal latencies makes every mixed-precision
 * evaluation end this way (the way this error path is tested).  The paper
 * has no counterpart of this entry point. */
int mera_set_device_wait(mera_t m, double seconds);

/* Device allocator for every buffer the library allocates (tensors, level
 * operators, Krylov vectors, workspaces, offset tables), process-wide.
 * alloc(bytes, user) returns device memory of at least `bytes` bytes,
 * aligned to 256 bytes, or NULL when it cannot: the call that needed the
 * memory then frees what it had allocated and returns MERA_ERR_OOM (the
 * server defers the admission of a request whose creation failed this way
 * while others run, and fails it only when it is alone).  dealloc(ptr,
 * user) takes back a pointer alloc returned.  alloc = NULL restores
 * cudaMalloc / cudaFree.  Every buffer is freed with the deallocator of the
 * allocator that made it.  Set it while no other thread is inside the
 * library.  Lets a caller route the library's memory through its own pool
 * (for example a framework's caching allocator) or bound it.  MERA_ERR_ARG
 * if alloc is set and dealloc is NULL.  The paper has no counterpart of
 * this entry point. */
typedef void* (*mera_alloc_fn)(size_t bytes, void* user);
typedef void (*mera_free_fn)(void* ptr, void* user);
int mera_set_allocator(mera_alloc_fn alloc, mera_free_fn dealloc, void* user);

/* Allocation-free batched dot products, for callers that cannot allocate
 * device memory (a host application that owns the whole GPU memory and
 * gives the library no allocator, or code that must not trigger the device
 * synchronisation of cudaMalloc).  Needs no mera_t; calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *   out[i] = sum_{j<n} X[i*ldx + j] * y[j],   i < k,
 * in the same fixed reduction order as the library's own dot products.
 * X, y: device pointers (doubles); out: host or device pointer to k doubles;
 * stream: a cudaStream_t (NULL = default stream); returns after the results
 * are in out.  Limits: 1 <= k <= 32 (MERA_ERR_ARG beyond), ldx >= n if k > 1.
 * Scratch: a fixed file-scope device array of 32*608+32 doubles (about
 * 152 KiB) held by every GPU that loads the library until exit.  The first
 * call on a device looks up that array's device address (make it before any
 * stream capture).  All calls share the array and it keeps the last call's
 * partial sums: calls whose work overlaps on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  Every call ends
 * with a synchronisation of `stream`.  A CUDA error left pending by an
 * earlier launch on the calling thread makes the call return MERA_ERR_CUDA
 * before it launches anything (the error stays pending).  The paper has no
 * counterpart of this entry point. */
int mera_dots_noalloc(const double* X, int64_t ldx, int k, const double* y, int64_t n, double* out,
                      void* stream);

const char* mera_strerror(int code);
const char* mera_last_error(mera_t m);

#ifdef __cplusplus
}
#endif
#endif /* MERA_H */
