// Internal declarations of libmera: the problem object (mera_ctx) and the
// functions its translation units share.  mera.cu: networks, energy and
// gradient, creation; mps.cu: the uniform MPS; geom.cu: preconditioner,
// retraction, transport; optim.cu: line search, L-BFGS, CG, Evenbly-Vidal;
// abi.cu: the C ABI.
#pragma once
#include "common.h"
#include "tn.h"
#include "tc_gemm.h"
#include "tnet.h"

#include <algorithm>
#include <exception>
#include <functional>
#include <memory>
#include <string>
#include <vector>

namespace mera {

struct Layer {
  int64_t cf = 0, cc = 0;
  std::unique_ptr<SideNet> net[2];
  SideBufs buf[2];
  std::vector<DevBuf> own[2];
  DevBuf amax[2];  // the sides' node maxima (scaled split-FP16)
  // ternary network: sides L, C, R
  std::unique_ptr<Net> tnet[3];
  NetBufs tbuf[3];
  std::vector<DevBuf> town[3];
};

// Per-evaluation results at one point.
struct Eval {
  double e = 0.0;
  DevBuf G;                       // projected gradient, all tensors concatenated
  DevBuf D;                       // partial derivatives
  std::vector<DevBuf> rho_v;      // per-tensor density matrices (preconditioner)
  std::vector<double> delta;      // |G_v|
  bool eig_ready = false;
  std::vector<DevBuf> evec, eval; // eigendecomposition of rho_v
  bool valid = false;
};

// Quantities of the low-rank exponential for one (point, direction, alpha).
struct StepGeom {
  bool valid = false;
  double alpha = 0.0;
  std::vector<DevBuf> Amat;   // u: A = W^T X ; w: V (evecs of X^T X)
  std::vector<DevBuf> E;      // u: exp(alpha A); Stiefel w: exp(alpha [[A, -P], [P, 0]]) (2p x 2p); else unused
  std::vector<DevBuf> Q2;     // Stiefel w: orthonormal basis of the range of (1 - W W^dag) X (n x p)
  std::vector<DevBuf> P1, P2, Pc;  // w: spectral matrices
};

}  // namespace mera

struct mera_ctx {
  mera_config cfg{};
  cudaStream_t s = nullptr;
  bool cplx = false;                      // interleaved complex128 data
  double hshift = 0.0;                    // evaluations use h3 - hshift 1 (Evenbly-Vidal sweeps)
  bool tern = false;                      // ternary network
  bool mps = false;                       // uniform MPS (one Grassmann tensor, two-site term)
  bool z2 = false;                        // Z2-symmetric problem: networks run by charge sector
  bool gnet = false;                      // networks on the data-defined executor (ternary; Z2 binary)
  int nsides = 2;                         // ascending maps per layer (3 ternary, 2 binary)
  int ns = 3;                             // sites of a level operator (3 binary, 2 ternary)
  int rs = 1;                             // reals per element (1 or 2)
  int L = 0, nt = 0;
  std::vector<int64_t> dims;
  std::vector<int64_t> rows, cols, offs;  // tensor shapes and offsets in a flat tangent
  int64_t total = 0;                      // flat tangent length
  mera::TablePool pool;
  std::vector<mera::Layer> layers;
  mera::DevBuf Wcur, Wtry;                // points (flat)
  mera::DevBuf h0;
  std::vector<mera::DevBuf> h, rho;       // level operators h_0..h_L, rho_0..rho_L
  mera::DevBuf x;                         // scale-invariant series
  mera::DevBuf bvec;                      // right-hand side 1/chi^3 of the fixed-point solve
  bool have_rho = false, have_x = false;
  mera::DevBuf kbasis, ktmp, kcoef;       // Krylov workspace
  mera::DevBuf scratch;                   // transient contraction buffers
  mera::DevBuf recomp;                    // N3, N7, N8 of every layer and side when recomputed (recompute_env)
  mera::Exec ex;                          // contraction arithmetic
  mera::DevBuf tc_ws, tc_err;             // tensor-core operand planes, wait-expiry flag
  mera::DevBuf tc_keep[2];                // packed planes of loop-invariant operands (sliced chain)
  // uniform MPS: two-site tensor B = A A, (h - e 1) B, its product with rho,
  // a (D d) x D scratch, the contracted terms h_l, h_r and the left
  // environment H_l (the right one lives in x, rho in rho[0])
  mera::DevBuf mB, mHB, mT, mA1, mhl, mhr, mHl;
  mera::GemmPlan mps_hplan;               // h on the physical pair of B
  mera::DevBuf gtmp[6];                   // geometry temporaries
  mera::Reducer red;
  mera::Eval ev[2];
  int cur = 0;                            // index of the current point's Eval
  mera::StepGeom geom;
  std::vector<mera::DevBuf> eig_cache;    // last eigenvectors of each rho_v (warm starts)
  mera::EigWork eigw;                      // Jacobi scratch
  std::vector<int> eig_uses;
  // optimiser
  std::vector<mera::DevBuf> mem_s, mem_y;
  std::vector<double> mem_rho;
  int mem_n = 0;
  mera::DevBuf dir, dir2, tmpv, tmpv2;
  double alpha_prev = 1.0;
  int iters = 0;
  mera::Prof prof;
  int64_t matvecs = 0;
  std::string err;
  // serving: evaluations go to the problem's cohort (same-configuration
  // problems evaluated together, group.cu) instead of running alone
  void (*cohort_eval)(void* cohort, mera_ctx& c, const double* W, mera::Eval& E) = nullptr;
  void* cohort = nullptr;
  int64_t evals_batched = 0;  // evaluations that ran together with other problems
};

namespace mera {

using Ctx = mera_ctx;

inline double* P(const DevBuf& b) { return b.as<double>(); }

inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}
// order of a level operator (matrix of ns sites of dimension c)
inline int64_t opn(const Ctx& c, int64_t dim) { return ipow(dim, c.ns); }

// Tensor i is a Grassmann point (an MPS tensor, or an isometry unless the
// config asks for Stiefel); the others (disentanglers, Stiefel isometries)
// use the Stiefel forms.
inline bool grass(const Ctx& c, int i) { return c.mps || (i % 2 == 1 && !c.cfg.w_stiefel); }

// element-type helpers: x = (x + x^dag)/2, x += a 1, matrix products whose
// 'C' operands are conjugate-transposed (plain transposes for real data)
inline void herm(Ctx& c, double* x, int64_t n, cudaStream_t s) {
  if (c.cplx) hermitize(x, n, s); else symmetrize(x, n, s);
}
inline void add_id(Ctx& c, double a, double* x, int64_t n, cudaStream_t s) {
  if (c.cplx) add_identity_c(a, 0.0, x, n, s); else add_identity(a, x, n, s);
}
inline void mm(Ctx& c, char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
               const double* B, int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t s) {
  gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, c.cplx);
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ---- mera.cu ----
// slice length of the middle coarse leg b of the chi^9 chain (0: unsliced)
int64_t choose_chunk(int64_t cf, int64_t cc);
// throws MERA_ERR_DEVICE_TIMEOUT (and clears the flag) if a bounded device wait expired
void check_device_flag(Ctx& c, cudaStream_t s);
// restarted GMRES for op(x) = b from the guess in x; returns the operator applications
int gmres(Ctx& c, const std::function<void(const double*, double*)>& op, const double* b, double* x, int64_t n,
          double tol, cudaStream_t s);
// G = the tangent projection of D at W (tensor i)
void project_tensor(Ctx& c, int i, const double* W, const double* D, double* G, cudaStream_t s);
// full evaluation at W into E; the energy alone
void energy_grad(Ctx& c, const double* W, Eval& E, cudaStream_t s);
double forward_energy(Ctx& c, const double* W, cudaStream_t s);
void check_isometric(Ctx& c, const double* W, cudaStream_t s);
std::vector<int> fused_charges(const std::vector<int64_t>& dims);
// legs (dimensions) of the rows and columns of tensor i of a MERA point
void tensor_legs(const Ctx& c, int i, std::vector<int64_t>& rows, std::vector<int64_t>& cols);
void check_z2_point(Ctx& c, const double* W, cudaStream_t s);
void create(Ctx& c, const mera_config& cfg, const void* h3, cudaStream_t s);
// why cfg's flags, tolerances or counts are out of range ("" if they are not)
std::string config_range_error(const mera_config& cfg);

// binds a side's leaves: operator op, disentangler u, isometry w (mera.cu)
void bind_leaves(Layer& ly, int side, const double* op, const double* u, const double* w);
// floor of the Krylov solves' relative residual in a precision mode
double krylov_floor(int prec);
// whether a GMRES cycle's residual estimate may end a solve (mixed modes)
bool trust_estimate(int prec);
// per-tensor density matrices of the preconditioner at the last evaluation
void compute_rho_v(Ctx& c, Eval& E, const double* W, cudaStream_t s);

// ---- group.cu ----
// Evaluations of nb problems (binary network, real tensors, the same
// configuration) in lockstep: cs[k] at point Ws[k] into Es[k] (the energy
// only when grad is false); every product is one batched launch over the
// members with the workspace and wait flag of ex, on stream s.  Member k's
// arithmetic is that of its evaluation alone.  errs[k] receives member k's
// failure (null when it succeeded); the others are unaffected by it.
void eval_group(Ctx* const* cs, const double* const* Ws, Eval* const* Es, int nb, bool grad, const Exec& ex,
                cudaStream_t s, std::exception_ptr* errs);
// the binary, real, unsliced problems whose evaluation runs in eval_group
bool grouped_eval(const Ctx& c);

// ---- mps.cu ----
double mps_energy(Ctx& c, const double* A, cudaStream_t s);
void mps_energy_grad(Ctx& c, const double* A, Eval& E, cudaStream_t s);
void create_mps(Ctx& c, int64_t* nS, int64_t* gmax);

// ---- geom.cu ----
// out[i] = f(ev[i]) for the spectral functions of geom.cu (kind as there)
void spectral_values(const double* ev, int n, int kind, double a, double d, double* out, cudaStream_t s);
// out = V diag(f) V^T (n x n)
void v_diag_vt(const double* V, const double* f, int n, double* out, cudaStream_t s);
void ensure_eig(Ctx& c, Eval& E, cudaStream_t s);
void precondition(Ctx& c, Eval& E, const double* W, const double* X, double* Xt, cudaStream_t s);
void polar_ns(Ctx& c, double* X, int64_t n, int64_t p, cudaStream_t s);
void make_geom(Ctx& c, const double* W, const double* X, double alpha, cudaStream_t s);
void apply_retract(Ctx& c, const double* W, const double* X, double* Wout, cudaStream_t s);
void apply_transport(Ctx& c, const double* W, const double* X, double* Y, cudaStream_t s);
double inner(Ctx& c, const double* X, const double* Y, cudaStream_t s);

// ---- optim.cu ----
void ensure_current(Ctx& c, cudaStream_t s);
void clear_history(Ctx& c);
void lbfgs_step(Ctx& c, mera_iter_info* info, cudaStream_t s);
void cg_step(Ctx& c, mera_iter_info* info, cudaStream_t s);
void gd_step(Ctx& c, mera_iter_info* info, cudaStream_t s);
void ev_sweep(Ctx& c, double gamma, mera_iter_info* info, cudaStream_t s);

}  // namespace mera
