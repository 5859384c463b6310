// The uniform MPS of Sec. 5 on libmera's geometry and optimisers: transfer
// maps, the fixed point, the energy and its partial derivative, and the
// problem's shapes and buffers.
#include "ctx.h"

#include <cmath>

namespace mera {
namespace {
// y += (re + i im) x, n interleaved complex elements
__global__ void axpy_c_k(double re, double im, const double2* __restrict__ x, double2* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 a = x[i];
  double2 b = y[i];
  b.x += re * a.x - im * a.y;
  b.y += re * a.y + im * a.x;
  y[i] = b;
}

}  // namespace

// ------------------------------------------------------------ uniform MPS --
// Sec. 5: one left-canonical tensor A ((D d) x D, rows (a s), column b; A^s
// the D x D matrix at fixed physical index s) on the Grassmann manifold and a
// two-site term h.  With the transfer maps
//   E_R(y) = sum_s A^s y A^s^dag,   E_L(x) = sum_s A^s^dag x A^s  (E_L(1) = 1),
// rho the unit-trace fixed point of E_R (Eq. mps_right_transfermatrix),
// B = A A the two-site tensor [a][s][t][c] and HB = h applied to its
// physical pair, the energy per site is e = Re <B, HB rho>.  The partial
// derivative of Eq. mps_derivative, D = 2 de/d conj(A), takes the shifted
// term h - e 1 (which makes the environment sums converge):
//   T   = (h - e) B rho,  h_l = B^dag (h - e) B,  h_r = T B^dag,
//   (1 - E_L + |1)(rho|) H_l = h_l,  (1 - E_R + |rho)(1|) H_r = h_r,
//   D/2 = T A^dag (bra copy on the left site of the term)
//       + A^dag T (bra copy on the right site) + H_l A rho + A H_r,
// the products read with the reshapes of the row-major arrays named below.

// out = beta out + alpha E_R(y)   (D x D; scratch mA1)
void mps_right(Ctx& c, const double* A, const double* y, double* out, double alpha, double beta, cudaStream_t s) {
  const int64_t D = c.cols[0], d = c.cfg.d_b;
  double* T = P(c.mA1);
  mm(c, 'N', 'N', D * d, D, D, 1.0, A, D, y, D, 0.0, T, D, s);                 // T[(a s), c] = (A^s y)[a, c]
  mm(c, 'N', 'C', D, D, d * D, alpha, T, d * D, A, d * D, beta, out, D, s);     // T[a, (s c)] A[e, (s c)]^*
}

// out = beta out + alpha E_L(x)   (D x D; scratch mA1)
void mps_left(Ctx& c, const double* A, const double* x, double* out, double alpha, double beta, cudaStream_t s) {
  const int64_t D = c.cols[0], d = c.cfg.d_b;
  double* T = P(c.mA1);
  mm(c, 'N', 'N', D, d * D, D, 1.0, x, D, A, d * D, 0.0, T, d * D, s);         // T[a, (s c)] = (x A^s)[a, c]
  mm(c, 'C', 'N', D, D, D * d, alpha, A, D, T, D, beta, out, D, s);             // A[(a s), b]^* T[(a s), c]
}

// Energy per site at A: rho (GMRES, warm-started), B, HB and mT = HB rho.
double mps_energy(Ctx& c, const double* A, cudaStream_t s) {
  const int64_t D = c.cols[0], d = c.cfg.d_b, n = D * D, nr = n * c.rs, nb = D * d * d * D * c.rs;
  double* rho = P(c.rho[0]);
  double* bvec = P(c.bvec);
  fill(0.0, bvec, nr, s);
  add_id(c, 1.0 / (double)D, bvec, D, s);
  if (!c.have_rho) copy(rho, bvec, nr, s);
  c.have_rho = false;  // valid again once the solve below has succeeded
  // (1 - E_R + |b)(1|) rho = b, b = 1/D: the fixed point with Tr rho = 1
  auto op_rho = [&](const double* v, double* out) {
    copy(out, v, nr, s);
    mps_right(c, A, v, out, -1.0, 1.0, s);
    if (c.cplx) {
      double tr, ti;
      c.red.trace_c(v, D, s, &tr, &ti);
      add_identity_c(tr / (double)D, ti / (double)D, out, D, s);
    } else {
      axpy(c.red.trace(v, D, s), bvec, out, n, s);
    }
    ++c.matvecs;
  };
  gmres(c, op_rho, bvec, rho, nr, c.cfg.krylov_tol, s);
  double tr = 0.0, ti = 0.0;
  if (c.cplx) c.red.trace_c(rho, D, s, &tr, &ti); else tr = c.red.trace(rho, D, s);
  if (!(std::fabs(tr) > 0)) throw Error(MERA_ERR_NONFINITE, "MPS fixed point has zero trace");
  scal(1.0 / tr, rho, nr, s);
  herm(c, rho, D, s);
  if (!std::isfinite(tr)) throw Error(MERA_ERR_NONFINITE, "MPS fixed point is not finite");
  c.have_rho = true;
  // B[(a s), (t c)] = A[(a s), b] A[b, (t c)]
  mm(c, 'N', 'N', D * d, d * D, D, 1.0, A, D, A, d * D, 0.0, P(c.mB), d * D, s);
  // HB[a, (s t), c] = h[(s t), (u v)] B[a, (u v), c]
  GettCall g = c.mps_hplan.proto;
  g.A = P(c.h0);
  g.B = P(c.mB);
  g.C = P(c.mHB);
  g.cplx = c.cplx;
  gett_f64(g, s);
  mm(c, 'N', 'N', D * d * d, D, D, 1.0, P(c.mHB), D, rho, D, 0.0, P(c.mT), D, s);  // HB rho
  // Tr T_h(rho) = sum conj(B) (HB rho): the real dot product of the arrays
  const double e = c.red.dot(P(c.mB), P(c.mT), nb, s);
  if (!std::isfinite(e)) throw Error(MERA_ERR_NONFINITE, "non-finite MPS energy");
  return e;
}

// Full MPS evaluation at A into E (energy, D, G, delta, rho for the preconditioner).
void mps_energy_grad(Ctx& c, const double* A, Eval& E, cudaStream_t s) {
  E.e = mps_energy(c, A, s);
  const int64_t D = c.cols[0], d = c.cfg.d_b, n = D * D, nr = n * c.rs, nb = D * d * d * D * c.rs;
  const double* rho = P(c.rho[0]);
  const double* B = P(c.mB);
  double* HB = P(c.mHB);
  double* T = P(c.mT);
  double* hl = P(c.mhl);
  double* hr = P(c.mhr);
  double* Hl = P(c.mHl);
  double* Hr = P(c.x);
  axpy(-E.e, B, HB, nb, s);                                                      // (h - e 1) B
  mm(c, 'N', 'N', D * d * d, D, D, 1.0, HB, D, rho, D, 0.0, T, D, s);           // T = (h - e) B rho
  mm(c, 'C', 'N', D, D, D * d * d, 1.0, B, D, HB, D, 0.0, hl, D, s);            // h_l = B^dag (h - e) B
  mm(c, 'N', 'C', D, D, d * d * D, 1.0, T, d * d * D, B, d * d * D, 0.0, hr, D, s);  // h_r = T B^dag
  if (!c.have_x) {
    copy(Hl, hl, nr, s);
    copy(Hr, hr, nr, s);
  }
  c.have_x = false;  // valid again once both solves below have succeeded
  // (1 - E_L + |1)(rho|) H_l = h_l: the added term is Tr(rho v) 1
  auto op_l = [&](const double* v, double* out) {
    copy(out, v, nr, s);
    mps_left(c, A, v, out, -1.0, 1.0, s);
    if (c.cplx) {
      double tr, ti;
      c.red.dot_c(rho, v, n, s, &tr, &ti);  // sum conj(rho_ij) v_ij = Tr(rho v), rho hermitian
      add_identity_c(tr, ti, out, D, s);
    } else {
      add_identity(c.red.dot(v, rho, n, s), out, D, s);
    }
    ++c.matvecs;
  };
  // (1 - E_R + |rho)(1|) H_r = h_r: the added term is Tr(v) rho
  auto op_r = [&](const double* v, double* out) {
    copy(out, v, nr, s);
    mps_right(c, A, v, out, -1.0, 1.0, s);
    if (c.cplx) {
      double tr, ti;
      c.red.trace_c(v, D, s, &tr, &ti);
      axpy_c_k<<<blocks(n), 256, 0, s>>>(tr, ti, reinterpret_cast<const double2*>(rho),
                                         reinterpret_cast<double2*>(out), n);
      count_launch();
      MERA_CHECK_LAUNCH();
    } else {
      axpy(c.red.trace(v, D, s), rho, out, n, s);
    }
    ++c.matvecs;
  };
  gmres(c, op_l, hl, Hl, nr, c.cfg.krylov_tol, s);
  gmres(c, op_r, hr, Hr, nr, c.cfg.krylov_tol, s);
  c.have_x = true;
  double* Dv = P(E.D);
  double* Arho = P(c.mA1);
  mm(c, 'N', 'C', D * d, D, d * D, 2.0, T, d * D, A, d * D, 0.0, Dv, D, s);      // T[(a s), (t c)] A[e, (t c)]^*
  mm(c, 'C', 'N', D, d * D, D * d, 2.0, A, D, T, d * D, 1.0, Dv, d * D, s);      // A[(e t), c]^* T[(e t), (s f)]
  mm(c, 'N', 'N', D * d, D, D, 1.0, A, D, rho, D, 0.0, Arho, D, s);             // A rho
  mm(c, 'N', 'N', D, d * D, D, 2.0, Hl, D, Arho, d * D, 1.0, Dv, d * D, s);     // H_l A rho
  mm(c, 'N', 'N', D * d, D, D, 2.0, A, D, Hr, D, 1.0, Dv, D, s);                // A H_r
  project_tensor(c, 0, A, Dv, P(E.G), s);
  const double* g = P(E.G);
  E.delta.assign(1, std::sqrt(c.red.dot(g, g, c.rows[0] * c.cols[0] * c.rs, s)));
  if (!std::isfinite(E.delta[0])) throw Error(MERA_ERR_NONFINITE, "non-finite MPS gradient");
  copy(P(E.rho_v[0]), rho, nr, s);
  E.eig_ready = false;
  E.valid = true;
}

// Shapes and buffers of a uniform MPS (Sec. 5): one (D d) x D tensor, the
// Krylov vectors and scratch of its D x D transfer-map solves.
void create_mps(Ctx& c, int64_t* nS, int64_t* gmax) {
  const mera_config& cfg = c.cfg;
  if (cfg.d_b < 2 || cfg.chi < 1 || cfg.n_trans != 0) throw Error(MERA_ERR_ARG, "MPS: d_b >= 2, chi >= 1, n_trans = 0");
  if (cfg.prec != MERA_PREC_FP64) throw Error(MERA_ERR_UNSUPPORTED, "the MPS runs in the FP64 path only");
  if (cfg.w_stiefel) throw Error(MERA_ERR_UNSUPPORTED, "the MPS tensor is a Grassmann point (right rotations are gauge)");
  const int64_t D = cfg.chi, d = cfg.d_b, es = sizeof(double) * c.rs;
  c.L = 0;
  c.dims.assign(1, D);
  c.nt = 1;
  c.rows.assign(1, D * d);
  c.cols.assign(1, D);
  c.offs.assign(1, 0);
  c.total = D * d * D * c.rs;
  c.rho.emplace_back(es * D * D);
  for (DevBuf* b : {&c.mB, &c.mHB, &c.mT}) b->alloc(es * D * d * d * D);
  c.mA1.alloc(es * D * d * D);
  for (DevBuf* b : {&c.mhl, &c.mhr, &c.mHl}) b->alloc(es * D * D);
  auto desc = [](std::vector<int> legs, std::vector<int64_t> ext) {
    TDesc t;
    t.legs = legs;
    t.ext = ext;
    t.stride.assign(legs.size(), 1);
    for (size_t j = legs.size(); j-- > 1;) t.stride[j - 1] = t.stride[j] * ext[j];
    return t;
  };
  enum { ls, lt, lu, lv, la, lc };
  // HB[a s t c] = h[s t u v] B[a u v c]
  c.mps_hplan = make_plan(desc({ls, lt, lu, lv}, {d, d, d, d}), desc({la, lu, lv, lc}, {D, d, d, D}),
                          desc({la, ls, lt, lc}, {D, d, d, D}), c.pool);
  *nS = D * D * c.rs;
  *gmax = D * d * D;  // the tensor (polar scratch); D x D matrices and 2D x 2D embeddings fit after the x4 below
}

}  // namespace mera
