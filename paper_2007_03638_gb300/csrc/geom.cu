// Geometry of the tensors' manifolds (Sec. 2.3, Sec. 3): the preconditioner,
// the exponential retraction and the vector transport in their low-rank
// forms, polar re-isometrisation, the inner product.
#include "ctx.h"

#include <cmath>

namespace mera {
namespace {
__global__ void vfvt_k(const double* __restrict__ V, const double* __restrict__ f, int n,
                       double* __restrict__ out) {
  // out = V diag(f) V^T  (n x n)
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  double s = 0.0;
  for (int k = 0; k < n; ++k) s = fma(V[(int64_t)i * n + k] * f[k], V[(int64_t)j * n + k], s);
  out[idx] = s;
}

// out_ij = 2 a_ij / (lt_i + lt_j)
__global__ void sylvester_scale_k(double* a, const double* __restrict__ lt, int n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  a[idx] = 2.0 * a[idx] / (lt[i] + lt[j]);
}

// evals -> function values used by the Grassmann retraction/transport and
// the preconditioner (kind: 0 cos(a s), 1 sin(a s)/s, 2 (1-cos(a s))/s^2,
// 3 1/sqrt(l^2+d^2), 4 sqrt(l^2+d^2), 5 1/sqrt(max(l, d)), 6 1/(l + d),
// 7 1/sqrt(l) for l > d else 0, 8 sqrt(max(l, 0))); for kinds 0-2 the input is s^2.
__global__ void spectral_k(const double* __restrict__ ev, int n, int kind, double a, double d,
                           double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l = ev[i];
  double r;
  if (kind <= 2) {
    const double s = sqrt(fmax(l, 0.0));
    const double x = a * s;
    if (kind == 0) {
      r = cos(x);
    } else if (kind == 1) {
      r = (fabs(x) < 1e-4) ? a * (1.0 - x * x / 6.0 + x * x * x * x / 120.0) : sin(x) / s;
    } else {
      r = (fabs(x) < 1e-4) ? a * a * (0.5 - x * x / 24.0 + x * x * x * x / 720.0)
                           : (1.0 - cos(x)) / (s * s);
    }
  } else if (kind == 3) {
    r = 1.0 / sqrt(l * l + d * d);
  } else if (kind == 4) {
    r = sqrt(l * l + d * d);
  } else if (kind == 5) {
    r = 1.0 / sqrt(fmax(l, d));  // inverse square root of a positive semidefinite matrix (floor d)
  } else if (kind == 6) {
    r = 1.0 / (l + d);           // (rho + d 1)^(-1), the MPS preconditioner
  } else if (kind == 7) {
    r = l > d ? 1.0 / sqrt(l) : 0.0;  // pseudo-inverse square root
  } else {
    r = sqrt(fmax(l, 0.0));
  }
  out[i] = r;
}

// dst[i * ldd + j] = alpha src[i * lds + j] for i < rows, j < cols; rs reals
// per element (1 real, 2 interleaved complex)
__global__ void copy_block_k(double* __restrict__ dst, int64_t ldd, const double* __restrict__ src, int64_t lds,
                             int64_t rows, int64_t cols, double alpha, int rs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols * rs) return;
  const int64_t e = idx / rs, part = idx % rs, i = e / cols, j = e % cols;
  dst[(i * ldd + j) * rs + part] = alpha * src[(i * lds + j) * rs + part];
}

}  // namespace

void spectral_values(const double* ev, int n, int kind, double a, double d, double* out, cudaStream_t s) {
  spectral_k<<<blocks(n), 256, 0, s>>>(ev, n, kind, a, d, out);
}

void v_diag_vt(const double* V, const double* f, int n, double* out, cudaStream_t s) {
  vfvt_k<<<blocks((int64_t)n * n), 256, 0, s>>>(V, f, n, out);
}

// Eigendecomposition of every rho_v.  Complex hermitian matrices are
// decomposed through their real symmetric embedding [[Re, -Im], [Im, Re]]
// (order 2p): any real function of the matrix is the embedding of the
// same function of the complex matrix.
void ensure_eig(Ctx& c, Eval& E, cudaStream_t s) {
  if (E.eig_ready) return;
  for (int i = 0; i < c.nt; ++i) {
    const int64_t p = c.cols[i], q = p * c.rs;  // order of the (embedded) problem
    const int64_t pair = c.prof.begin(q, q, 0, s);
    double* A = P(c.gtmp[0]);
    double* src = P(E.rho_v[i]);
    if (c.cplx) {
      embed_complex(P(E.rho_v[i]), p, P(c.gtmp[4]), s);
      src = P(c.gtmp[4]);
    }
    if (q > 64 && c.eig_uses[i] > 0 && c.eig_uses[i] < 25) {
      // warm start: rotate rho into the previous eigenbasis, which leaves it
      // nearly diagonal, and continue the Jacobi sweeps from there
      double* T = P(c.gtmp[1]);
      double* Vc = P(c.eig_cache[i]);
      gemm_f64('N', 'N', q, q, q, 1.0, src, q, Vc, q, 0.0, T, q, s);
      gemm_f64('T', 'N', q, q, q, 1.0, Vc, q, T, q, 0.0, A, q, s);
      copy(P(E.evec[i]), Vc, q * q, s);
      sym_eig_from(A, P(E.evec[i]), P(E.eval[i]), (int)q, true, c.eigw, s);
      c.eig_uses[i]++;
    } else {
      copy(A, src, q * q, s);
      sym_eig(A, P(E.evec[i]), P(E.eval[i]), (int)q, c.eigw, s);
      c.eig_uses[i] = 1;
    }
    if (q > 64) copy(P(c.eig_cache[i]), P(E.evec[i]), q * q, s);
    c.prof.end(pair, 9300, s);
  }
  E.eig_ready = true;
}

// Xt = preconditioned X (per tensor), with E's density matrices and deltas.
void precondition(Ctx& c, Eval& E, const double* W, const double* X, double* Xt, cudaStream_t s) {
  if (!c.cfg.precond) {
    if (Xt != X) copy(Xt, X, c.total, s);
    return;
  }
  ensure_eig(c, E, s);
  for (int i = 0; i < c.nt; ++i) {
    const int64_t n = c.rows[i], p = c.cols[i], q = p * c.rs;
    const double* Wi = W + c.offs[i];
    const double* Xi = X + c.offs[i];
    double* Yi = Xt + c.offs[i];
    const double* V = P(E.evec[i]);
    double* lt = P(c.gtmp[5]);
    const bool stiefel = !grass(c, i);
    double* A = P(c.gtmp[0]);
    double* T = P(c.gtmp[1]);
    double* Rinv = P(c.gtmp[2]);
    double* Z = P(c.gtmp[3]);
    double* Em = P(c.gtmp[4]);
    // regularised inverse (rho^2 + delta^2)^(-1/2) = V diag(lt) V^T; for an
    // MPS (rho + delta^2 1)^(-1) (Sec. 5, delta = |G|)
    if (c.mps)
      spectral_k<<<blocks(q), 256, 0, s>>>(P(E.eval[i]), (int)q, 6, 0.0, E.delta[i] * E.delta[i], lt);
    else
      spectral_k<<<blocks(q), 256, 0, s>>>(P(E.eval[i]), (int)q, 3, 0.0, E.delta[i], lt);
    vfvt_k<<<blocks(q * q), 256, 0, s>>>(V, lt, (int)q, c.cplx ? Em : Rinv);
    count_launch(2);
    if (c.cplx) extract_complex(Em, p, Rinv, s);
    if (stiefel) {
      mm(c, 'C', 'N', p, p, n, 1.0, Wi, p, Xi, p, 0.0, A, p, s);   // A = W^dag X
      // Z = X - W A  (W_perp B part)
      copy(Z, Xi, n * p * c.rs, s);
      mm(c, 'N', 'N', n, p, p, -1.0, Wi, p, A, p, 1.0, Z, p, s);
      // At = V [2 (V^T A V)_ij / (lt_i + lt_j)] V^T  (on the embedding for complex data)
      spectral_k<<<blocks(q), 256, 0, s>>>(P(E.eval[i]), (int)q, 4, 0.0, E.delta[i], lt);
      count_launch();
      const double* Ain = A;
      if (c.cplx) {
        embed_complex(A, p, Em, s);
        Ain = Em;
      }
      gemm_f64('T', 'N', q, q, q, 1.0, V, q, Ain, q, 0.0, T, q, s);
      double* U2 = c.cplx ? Em : A;
      gemm_f64('N', 'N', q, q, q, 1.0, T, q, V, q, 0.0, U2, q, s);
      sylvester_scale_k<<<blocks(q * q), 256, 0, s>>>(U2, lt, (int)q);
      count_launch();
      gemm_f64('N', 'N', q, q, q, 1.0, V, q, U2, q, 0.0, T, q, s);
      if (c.cplx) {
        gemm_f64('N', 'T', q, q, q, 1.0, T, q, V, q, 0.0, Em, q, s);
        extract_complex(Em, p, A, s);
      } else {
        gemm_f64('N', 'T', q, q, q, 1.0, T, q, V, q, 0.0, A, q, s);
      }
      // Yi = W At + Z Rinv
      mm(c, 'N', 'N', n, p, p, 1.0, Wi, p, A, p, 0.0, Yi, p, s);
      mm(c, 'N', 'N', n, p, p, 1.0, Z, p, Rinv, p, 1.0, Yi, p, s);
    } else {
      mm(c, 'N', 'N', n, p, p, 1.0, Xi, p, Rinv, p, 0.0, Yi, p, s);
    }
  }
  MERA_CHECK_LAUNCH();
}

// ----------------------------------------------------------- geometry ------
void expm_skew(Ctx& c, const double* A, double alpha, int64_t n, double* E, double* T1, double* T2,
               cudaStream_t s) {
  // scaling and squaring with a degree-16 Taylor polynomial (Horner form)
  const int64_t nr = n * n * c.rs;
  const double nrm = std::fabs(alpha) * std::sqrt(c.red.dot(A, A, nr, s));
  int sq = 0;
  while (nrm / std::ldexp(1.0, sq) > 0.5) ++sq;
  const double a = alpha / std::ldexp(1.0, sq);
  const int q = 16;
  // T1 = I + a A / q
  axpby(a / q, A, 0.0, T1, nr, s);
  add_id(c, 1.0, T1, n, s);
  for (int k = q - 1; k >= 1; --k) {
    mm(c, 'N', 'N', n, n, n, a / k, A, n, T1, n, 0.0, T2, n, s);
    add_id(c, 1.0, T2, n, s);
    std::swap(T1, T2);
  }
  for (int k = 0; k < sq; ++k) {
    mm(c, 'N', 'N', n, n, n, 1.0, T1, n, T1, n, 0.0, T2, n, s);
    std::swap(T1, T2);
  }
  copy(E, T1, nr, s);
}

// Newton-Schulz polar iteration X <- X (3 - X^dag X)/2, in place (n x p).
void polar_ns(Ctx& c, double* X, int64_t n, int64_t p, cudaStream_t s) {
  double* S = P(c.gtmp[0]);
  double* Y = P(c.gtmp[1]);
  for (int it = 0; it < 2; ++it) {
    mm(c, 'C', 'N', p, p, n, -0.5, X, p, X, p, 0.0, S, p, s);
    add_id(c, 1.5, S, p, s);
    mm(c, 'N', 'N', n, p, p, 1.0, X, p, S, p, 0.0, Y, p, s);
    copy(X, Y, n * p * c.rs, s);
  }
}

// Non-square Stiefel point (an isometry with w_stiefel): Eq. retraction on
// the span of W and Q2, an orthonormal basis of the range of
// Z = (1 - W W^dag) X = W_perp B.  With A = W^dag X, Z^dag Z = V S^2 V^dag,
// Q2 = Z V S^-1 V^dag (directions with S = 0 dropped: they do not enter) and
// P = V S V^dag (so Z = Q2 P), e^{alpha Q_X} acts on [W Q2] as
// E = exp(alpha [[A, -P], [P, 0]]) and as the identity on the complement:
// R = W E11 + Q2 E21 and T(Y) = Y + [W Q2] (E - 1) [W Q2]^dag Y.  Leaves A in
// Amat, Q2 and E in the step geometry.
void stiefel_geom(Ctx& c, int i, const double* Wi, const double* Xi, double alpha, cudaStream_t s) {
  StepGeom& g = c.geom;
  const int64_t n = c.rows[i], p = c.cols[i], q = p * c.rs, p2 = 2 * p;
  double* A = P(g.Amat[i]);
  double* Q2 = P(g.Q2[i]);
  double* Z = P(c.gtmp[3]);
  double* ZZ = P(c.gtmp[0]);
  double* V = P(c.gtmp[1]);
  double* Pm = P(c.gtmp[2]);
  double* F = P(c.gtmp[4]);
  double* ev = P(c.gtmp[5]);
  mm(c, 'C', 'N', p, p, n, 1.0, Wi, p, Xi, p, 0.0, A, p, s);   // A = W^dag X
  copy(Z, Xi, n * p * c.rs, s);
  mm(c, 'N', 'N', n, p, p, -1.0, Wi, p, A, p, 1.0, Z, p, s);   // Z = X - W A
  const double zn = c.red.dot(Z, Z, n * p * c.rs, s);
  mm(c, 'C', 'N', p, p, n, 1.0, Z, p, Z, p, 0.0, ZZ, p, s);    // Z^dag Z
  herm(c, ZZ, p, s);
  if (c.cplx) {
    embed_complex(ZZ, p, F, s);
    copy(ZZ, F, q * q, s);
  }
  sym_eig(ZZ, V, ev, (int)q, c.eigw, s);
  // Q2 = Z V S^-1 V^dag (eigenvalues below 1e-24 |Z|^2 dropped), P = V S V^dag
  double* f = P(c.gtmp[2]);
  spectral_k<<<blocks(q), 256, 0, s>>>(ev, (int)q, 7, 0.0, 1e-24 * zn, f);
  vfvt_k<<<blocks(q * q), 256, 0, s>>>(V, f, (int)q, F);
  count_launch(2);
  MERA_CHECK_LAUNCH();
  double* Sinv = P(c.gtmp[0]);  // Z^dag Z is no longer needed
  if (c.cplx) extract_complex(F, p, Sinv, s); else copy(Sinv, F, q * q, s);
  mm(c, 'N', 'N', n, p, p, 1.0, Z, p, Sinv, p, 0.0, Q2, p, s);
  spectral_k<<<blocks(q), 256, 0, s>>>(ev, (int)q, 8, 0.0, 0.0, f);
  vfvt_k<<<blocks(q * q), 256, 0, s>>>(V, f, (int)q, F);
  count_launch(2);
  MERA_CHECK_LAUNCH();
  if (c.cplx) extract_complex(F, p, Pm, s); else copy(Pm, F, q * q, s);
  // M = [[A, -P], [P, 0]] (2p x 2p) in V's buffer, E = exp(alpha M)
  double* M = V;
  fill(0.0, M, p2 * p2 * c.rs, s);
  const unsigned nb = blocks(p * p * c.rs);
  copy_block_k<<<nb, 256, 0, s>>>(M, p2, A, p, p, p, 1.0, c.rs);
  copy_block_k<<<nb, 256, 0, s>>>(M + p * c.rs, p2, Pm, p, p, p, -1.0, c.rs);
  copy_block_k<<<nb, 256, 0, s>>>(M + p * p2 * c.rs, p2, Pm, p, p, p, 1.0, c.rs);
  count_launch(3);
  MERA_CHECK_LAUNCH();
  expm_skew(c, M, alpha, p2, P(g.E[i]), P(c.gtmp[4]), P(c.gtmp[5]), s);
}

// Fill c.geom for direction X at point W and step alpha.
void make_geom(Ctx& c, const double* W, const double* X, double alpha, cudaStream_t s) {
  StepGeom& g = c.geom;
  g.alpha = alpha;
  for (int i = 0; i < c.nt; ++i) {
    const int64_t n = c.rows[i], p = c.cols[i], q = p * c.rs;
    const double* Wi = W + c.offs[i];
    const double* Xi = X + c.offs[i];
    if (n == p) {
      mm(c, 'C', 'N', p, p, n, 1.0, Wi, p, Xi, p, 0.0, P(g.Amat[i]), p, s);
      expm_skew(c, P(g.Amat[i]), alpha, p, P(g.E[i]), P(c.gtmp[2]), P(c.gtmp[3]), s);
    } else if (grass(c, i)) {
      // Grassmann: X^dag X = V S^2 V^dag (through the real embedding for complex data)
      double* Z = P(c.gtmp[0]);
      double* ev = P(c.gtmp[5]);
      mm(c, 'C', 'N', p, p, n, 1.0, Xi, p, Xi, p, 0.0, Z, p, s);
      if (c.cplx) {
        embed_complex(Z, p, P(c.gtmp[4]), s);
        copy(Z, P(c.gtmp[4]), q * q, s);
      }
      sym_eig(Z, P(g.Amat[i]), ev, (int)q, c.eigw, s);
      double* f = P(c.gtmp[1]);
      double* F = P(c.gtmp[4]);
      for (int kind = 0; kind < 3; ++kind) {
        double* out = kind == 0 ? P(g.Pc[i]) : kind == 1 ? P(g.P1[i]) : P(g.P2[i]);
        spectral_k<<<blocks(q), 256, 0, s>>>(ev, (int)q, kind, alpha, 0.0, f);
        vfvt_k<<<blocks(q * q), 256, 0, s>>>(P(g.Amat[i]), f, (int)q, c.cplx ? F : out);
        count_launch(2);
        if (c.cplx) extract_complex(F, p, out, s);
      }
      MERA_CHECK_LAUNCH();
    } else {
      stiefel_geom(c, i, Wi, Xi, alpha, s);
    }
  }
  g.valid = true;
}

// Wout = R_W(X, alpha) (re-isometrised); uses c.geom.
void apply_retract(Ctx& c, const double* W, const double* X, double* Wout, cudaStream_t s) {
  StepGeom& g = c.geom;
  for (int i = 0; i < c.nt; ++i) {
    const int64_t n = c.rows[i], p = c.cols[i];
    const double* Wi = W + c.offs[i];
    const double* Xi = X + c.offs[i];
    double* Ri = Wout + c.offs[i];
    if (n == p) {
      mm(c, 'N', 'N', n, p, p, 1.0, Wi, p, P(g.E[i]), p, 0.0, Ri, p, s);
    } else if (grass(c, i)) {
      mm(c, 'N', 'N', n, p, p, 1.0, Wi, p, P(g.Pc[i]), p, 0.0, Ri, p, s);
      mm(c, 'N', 'N', n, p, p, 1.0, Xi, p, P(g.P1[i]), p, 1.0, Ri, p, s);
    } else {
      // R = W E11 + Q2 E21 (E is 2p x 2p)
      const double* E = P(g.E[i]);
      mm(c, 'N', 'N', n, p, p, 1.0, Wi, p, E, 2 * p, 0.0, Ri, p, s);
      mm(c, 'N', 'N', n, p, p, 1.0, P(g.Q2[i]), p, E + 2 * p * p * c.rs, 2 * p, 1.0, Ri, p, s);
    }
    polar_ns(c, Ri, n, p, s);
  }
}

// Y <- T_W(Y, X, alpha), in place; uses c.geom.
void apply_transport(Ctx& c, const double* W, const double* X, double* Y, cudaStream_t s) {
  StepGeom& g = c.geom;
  for (int i = 0; i < c.nt; ++i) {
    const int64_t n = c.rows[i], p = c.cols[i];
    const double* Wi = W + c.offs[i];
    const double* Xi = X + c.offs[i];
    double* Yi = Y + c.offs[i];
    double* Z = P(c.gtmp[0]);
    double* Z2 = P(c.gtmp[1]);
    if (n == p) {
      // W exp(aA) W^dag Y
      mm(c, 'C', 'N', p, p, n, 1.0, Wi, p, Yi, p, 0.0, Z, p, s);
      mm(c, 'N', 'N', p, p, p, 1.0, P(g.E[i]), p, Z, p, 0.0, Z2, p, s);
      mm(c, 'N', 'N', n, p, p, 1.0, Wi, p, Z2, p, 0.0, Yi, p, s);
    } else if (grass(c, i)) {
      // Y - W P1 (X^dag Y) - X P2 (X^dag Y)
      mm(c, 'C', 'N', p, p, n, 1.0, Xi, p, Yi, p, 0.0, Z, p, s);
      mm(c, 'N', 'N', p, p, p, 1.0, P(g.P1[i]), p, Z, p, 0.0, Z2, p, s);
      mm(c, 'N', 'N', n, p, p, -1.0, Wi, p, Z2, p, 1.0, Yi, p, s);
      mm(c, 'N', 'N', p, p, p, 1.0, P(g.P2[i]), p, Z, p, 0.0, Z2, p, s);
      mm(c, 'N', 'N', n, p, p, -1.0, Xi, p, Z2, p, 1.0, Yi, p, s);
    } else {
      // Y + W ((E11 - 1) C1 + E12 C2) + Q2 (E21 C1 + (E22 - 1) C2), C1 = W^dag Y, C2 = Q2^dag Y
      const double* E = P(g.E[i]);
      const double* Q2 = P(g.Q2[i]);
      const int64_t r = c.rs, ld = 2 * p;
      double* K1 = P(c.gtmp[2]);
      double* K2 = P(c.gtmp[3]);
      mm(c, 'C', 'N', p, p, n, 1.0, Wi, p, Yi, p, 0.0, Z, p, s);
      mm(c, 'C', 'N', p, p, n, 1.0, Q2, p, Yi, p, 0.0, Z2, p, s);
      mm(c, 'N', 'N', p, p, p, 1.0, E, ld, Z, p, 0.0, K1, p, s);
      axpy(-1.0, Z, K1, p * p * r, s);
      mm(c, 'N', 'N', p, p, p, 1.0, E + p * r, ld, Z2, p, 1.0, K1, p, s);
      mm(c, 'N', 'N', p, p, p, 1.0, E + p * ld * r, ld, Z, p, 0.0, K2, p, s);
      mm(c, 'N', 'N', p, p, p, 1.0, E + (p * ld + p) * r, ld, Z2, p, 1.0, K2, p, s);
      axpy(-1.0, Z2, K2, p * p * r, s);
      mm(c, 'N', 'N', n, p, p, 1.0, Wi, p, K1, p, 1.0, Yi, p, s);
      mm(c, 'N', 'N', n, p, p, 1.0, Q2, p, K2, p, 1.0, Yi, p, s);
    }
  }
}

double inner(Ctx& c, const double* X, const double* Y, cudaStream_t s) {
  return c.red.dot(X, Y, c.total, s);
}

}  // namespace mera
