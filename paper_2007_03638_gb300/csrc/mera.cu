// libmera: scale-invariant binary MERA energy/gradient and the Riemannian
// optimisation step on one GPU (FP64 path).
//
//   energy_grad   (Sec. 4, App. B)
//     up-sweep    h_{l+1} = (A_L + A_R)(h_l)/2 through the transition layers
//     fixed point rho_S:  (1 - Dbar_S + |b><1|) rho = b, b = 1/chi^3, GMRES
//     series      x (1 - A') = <h_L|:  x - Abar_S(x) + Tr(x rho_S) 1 = h_L, GMRES
//     down-sweep  reverse pass of Tr(Abar_l(h_l) rho_{l+1}) per layer gives
//                 rho_l and the environments; the scale-invariant layer uses
//                 Tr(Abar_S(x) rho_S)
//     projection  Eqs. (stiefel_gradient), (grassmann_gradient)
//   geometry      retraction / transport (Eqs. retraction, transport) with the
//                 low-rank forms: W exp(alpha W^dag X) for unitaries, sines and
//                 cosines of the singular values of X for Grassmann tangents;
//                 polar re-isometrisation by Newton-Schulz
//   preconditioner Eq. (preconditioner_solution) in the eigenbasis of rho_v
//   optimiser     L-BFGS two-loop / Hager-Zhang CG, Hager-Zhang line search
#include "common.h"
#include "tn.h"
#include "tc_gemm.h"
#include "tnet.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>

namespace mera {
thread_local Prof* g_prof = nullptr;

namespace {

// ------------------------------------------------------------ kernels -----
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

// rho_w of the ternary network: the one-site marginal (Tr_right + Tr_left) / 2
// of a two-site operator r (c states per site, row-major (c^2 x c^2)).
__global__ void marg_tern_k(const double* __restrict__ r, int64_t c, double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c * c) return;
  const int64_t a = idx / c, A = idx % c, n = c * c;
  double s = 0.0;
  for (int64_t b = 0; b < c; ++b) s += r[(a * c + b) * n + A * c + b] + r[(b * c + a) * n + b * c + A];
  out[idx] = 0.5 * s;
}
__global__ void marg_tern_c_k(const double2* __restrict__ r, int64_t c, double2* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c * c) return;
  const int64_t a = idx / c, A = idx % c, n = c * c;
  double sx = 0.0, sy = 0.0;
  for (int64_t b = 0; b < c; ++b) {
    const double2 u = r[(a * c + b) * n + A * c + b], v = r[(b * c + a) * n + b * c + A];
    sx += u.x + v.x;
    sy += u.y + v.y;
  }
  out[idx] = make_double2(0.5 * sx, 0.5 * sy);
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

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

// ===================================================================== ctx ==
struct Layer {
  int64_t cf = 0, cc = 0;
  std::unique_ptr<SideNet> net[2];
  SideBufs buf[2];
  std::vector<DevBuf> own[2];
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
  bool z2 = false;                        // Z2-symmetric ternary problem: networks run by charge sector
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
};

namespace mera {
namespace {

using Ctx = mera_ctx;

double* P(const DevBuf& b) { return b.as<double>(); }

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}
// order of a level operator (matrix of ns sites of dimension c)
int64_t opn(const Ctx& c, int64_t dim) { return ipow(dim, c.ns); }

// Tensor i is a Grassmann point (an MPS tensor, or an isometry unless the
// config asks for Stiefel); the others (disentanglers, Stiefel isometries)
// use the Stiefel forms.
bool grass(const Ctx& c, int i) { return c.mps || (i % 2 == 1 && !c.cfg.w_stiefel); }

// element-type helpers: x = (x + x^dag)/2, x += a 1, matrix products whose
// 'C' operands are conjugate-transposed (plain transposes for real data)
void herm(Ctx& c, double* x, int64_t n, cudaStream_t s) {
  if (c.cplx) hermitize(x, n, s); else symmetrize(x, n, s);
}
void add_id(Ctx& c, double a, double* x, int64_t n, cudaStream_t s) {
  if (c.cplx) add_identity_c(a, 0.0, x, n, s); else add_identity(a, x, n, s);
}
void mm(Ctx& c, char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
        const double* B, int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t s) {
  gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, c.cplx);
}

// ------------------------------------------------------ network binding ----
void bind_leaves(Layer& ly, int side, const double* op, const double* u, const double* w) {
  SideBufs& b = ly.buf[side];
  b.leaf[0] = op;
  for (int l : {1, 2, 3, 5}) b.leaf[l] = u;
  for (int l : {4, 6, 7, 8, 9, 10}) b.leaf[l] = w;
}

// Slice length of the coarse leg b: keep the 7-leg intermediate (chi_f^6 * b
// entries) at most 2^30 entries per slice.
int64_t choose_chunk(int64_t cf, int64_t cc) {
  const int64_t f6 = ipow(cf, 6);
  if (f6 * cc <= (int64_t)1 << 30) return 0;
  int64_t nb = 1;
  for (int64_t d = 1; d <= cc; ++d)
    if (cc % d == 0 && f6 * d <= (int64_t)1 << 30) nb = d;
  return nb;
}

// Ternary network: three networks per layer, every internal node value and
// adjoint in its own buffer (no intermediate above chi^6).
void build_layers_ternary(Ctx& c) {
  const bool mixed = c.cfg.prec != MERA_PREC_FP64;
  const size_t es = (mixed ? sizeof(float) : sizeof(double)) * c.rs;
  size_t ws_need = 0;
  for (int l = 0; l <= c.L; ++l) {
    Layer& ly = c.layers[l];
    ly.cf = c.dims[l];
    ly.cc = l < c.L ? c.dims[l + 1] : c.dims[l];
    for (int sd = 0; sd < 3; ++sd) {
      ly.tnet[sd] = std::make_unique<Net>(ternary_netdef("LCR"[sd]), ly.cf, ly.cc, c.pool, c.z2);
      Net& net = *ly.tnet[sd];
      NetBufs& b = ly.tbuf[sd];
      b.leaf.assign(net.nleaf(), nullptr);
      b.val.assign(net.nnode(), nullptr);
      b.adj.assign(net.nnode(), nullptr);
      for (int node = net.nleaf(); node < net.nnode(); ++node) {
        if (node != net.root()) {
          ly.town[sd].emplace_back(es * net.size(node));
          b.val[node] = P(ly.town[sd].back());
        }
        ly.town[sd].emplace_back(es * net.size(node));
        b.adj[node] = P(ly.town[sd].back());
      }
      // charge sectors leave the odd-charge entries of node buffers untouched
      // (and never read them): keep those at zero
      if (c.z2)
        for (DevBuf& db : ly.town[sd]) MERA_CUDA(cudaMemsetAsync(db.p, 0, db.bytes, c.s));
      b.f32 = mixed;
      b.cplx = c.cplx;
      b.ex = &c.ex;
      for (const GemmPlan* p : net.plans()) ws_need = std::max(ws_need, tc_workspace_bytes(p->proto, c.cfg.prec));
    }
  }
  c.ex.prec = c.cfg.prec;
  if (mixed) {
    c.tc_ws.alloc(ws_need);
    c.tc_err.alloc(sizeof(int));
    MERA_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.s));
    MERA_CUDA(cudaStreamSynchronize(c.s));
    c.ex.ws = c.tc_ws.p;
    c.ex.ws_bytes = ws_need;
    c.ex.err = c.tc_err.as<int>();
  }
}

void bind_ternary(Layer& ly, int sd, const double* op, const double* u, const double* w) {
  NetBufs& b = ly.tbuf[sd];
  const Net& net = *ly.tnet[sd];
  for (int i = 0; i < net.nleaf(); ++i) {
    const int r = net.role(i);
    b.leaf[i] = r == ROLE_OP ? op : (r == ROLE_U || r == ROLE_UB) ? u : w;
  }
}

void build_layers(Ctx& c) {
  c.layers.resize(c.L + 1);
  if (c.tern) {
    build_layers_ternary(c);
    return;
  }
  const bool mixed = c.cfg.prec != MERA_PREC_FP64;
  const size_t es = (mixed ? sizeof(float) : sizeof(double)) * c.rs;
  size_t scratch_need = 0, ws_need = 0, kneed[2] = {0, 0};
  // With recomputation, the operator-dependent nodes N3, N7, N8 are rebuilt
  // by each side's forward pass right before they are read (the sides and
  // layers run one after another on the stream): one set serves all.
  const bool share = c.cfg.recompute_env != 0;
  const int dep[3] = {13, 17, 18};
  int64_t dep_max[3] = {0, 0, 0};
  for (int l = 0; l <= c.L; ++l) {
    Layer& ly = c.layers[l];
    ly.cf = c.dims[l];
    ly.cc = l < c.L ? c.dims[l + 1] : c.dims[l];
    int64_t chunk = choose_chunk(ly.cf, ly.cc);
    if (c.cfg.b_chunk > 0) {
      if (ly.cc % c.cfg.b_chunk) throw Error(MERA_ERR_ARG, "b_chunk must divide every coarse bond dimension");
      chunk = c.cfg.b_chunk < ly.cc ? c.cfg.b_chunk : 0;
    }
    for (int sd = 0; sd < 2; ++sd) {
      ly.net[sd] = std::make_unique<SideNet>(sd == 0 ? 'L' : 'R', ly.cf, ly.cc, c.pool, chunk);
      SideNet& net = *ly.net[sd];
      // persistent node values: N1 N3 N4 N6 N7 N8 N9 (N3 N7 N8 shared when recomputed)
      for (int node : {11, 13, 14, 16, 17, 18, 19}) {
        if (share && (node == 13 || node == 17 || node == 18)) {
          const int k = node == 13 ? 0 : node == 17 ? 1 : 2;
          dep_max[k] = std::max(dep_max[k], net.alloc_size(node));
          continue;
        }
        ly.own[sd].emplace_back(es * net.alloc_size(node));
        ly.buf[sd].val[node] = P(ly.own[sd].back());
      }
      ly.buf[sd].f32 = mixed;
      ly.buf[sd].cplx = c.cplx;
      ly.buf[sd].ex = &c.ex;
      size_t need = 0;
      for (int node : {12, 15}) need += net.alloc_size(node);
      for (int node = 11; node < 20; ++node) need += net.alloc_size(node);
      scratch_need = std::max(scratch_need, need);
      for (const GemmPlan* p : net.executed_plans())
        ws_need = std::max(ws_need, tc_workspace_bytes(p->proto, c.cfg.prec));
      size_t kn[2];
      keep_need(net, c.cfg.prec, kn);
      kneed[0] = std::max(kneed[0], kn[0]);
      kneed[1] = std::max(kneed[1], kn[1]);
    }
  }
  c.scratch.alloc(es * scratch_need);
  if (share) {
    // each part aligned like a separate allocation (the tensor-core epilogue
    // picks its store path, and with it its rounding, from the alignment)
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    c.recomp.alloc(al(es * dep_max[0]) + al(es * dep_max[1]) + al(es * dep_max[2]));
    for (int l = 0; l <= c.L; ++l)
      for (int sd = 0; sd < 2; ++sd) {
        char* p = static_cast<char*>(c.recomp.p);
        for (int k = 0; k < 3; ++k) {
          c.layers[l].buf[sd].val[dep[k]] = reinterpret_cast<double*>(p);
          p += al(es * dep_max[k]);
        }
      }
  }
  c.ex.prec = c.cfg.prec;
  if (mixed) {
    c.tc_ws.alloc(ws_need);
    c.tc_err.alloc(sizeof(int));
    MERA_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.s));
    MERA_CUDA(cudaStreamSynchronize(c.s));
    c.ex.ws = c.tc_ws.p;
    c.ex.ws_bytes = ws_need;
    for (int k = 0; k < 2; ++k)
      if (kneed[k]) {
        c.tc_keep[k].alloc(kneed[k]);
        c.ex.keep[k] = c.tc_keep[k].p;
        c.ex.keep_bytes[k] = kneed[k];
      }
    c.ex.err = c.tc_err.as<int>();
  }
  for (int l = 0; l <= c.L; ++l)
    for (int sd = 0; sd < 2; ++sd) {
      Layer& ly = c.layers[l];
      SideNet& net = *ly.net[sd];
      char* p = static_cast<char*>(c.scratch.p);
      for (int node : {12, 15}) {
        ly.buf[sd].val[node] = reinterpret_cast<double*>(p);
        p += es * net.alloc_size(node);
      }
      for (int node = 11; node < 20; ++node) {
        ly.buf[sd].adj[node] = reinterpret_cast<double*>(p);
        p += es * net.alloc_size(node);
      }
    }
}

void check_device_flag(Ctx& c, cudaStream_t s) {
  if (!c.tc_err.p) return;
  int e = 0;
  MERA_CUDA(cudaMemcpyAsync(&e, c.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  if (e) {
    MERA_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), s));
    throw Error(MERA_ERR_DEVICE_TIMEOUT, "tensor-core contraction: a bounded device-side wait expired");
  }
}

// -------------------------------------------------------- superoperators ---
// out = ao * out + af * Abar(op) (both sides), using layer l's tensors from point W.
void ascend(Ctx& c, int l, const double* W, const double* op, double* out, double af, cudaStream_t s) {
  Layer& ly = c.layers[l];
  const double* u = W + c.offs[2 * l];
  const double* w = W + c.offs[2 * l + 1];
  if (c.tern) {  // Abar = (A_L + A_C + A_R) / 3
    for (int sd = 0; sd < 3; ++sd) {
      bind_ternary(ly, sd, op, u, w);
      net_forward(*ly.tnet[sd], ly.tbuf[sd], out, af / 3.0, 1.0, s);
    }
    return;
  }
  for (int sd = 0; sd < 2; ++sd) {
    bind_leaves(ly, sd, op, u, w);
    side_forward(*ly.net[sd], ly.buf[sd], out, 0.5 * af, 1.0, s);
  }
}

void prepare_layer(Ctx& c, int l, const double* W, cudaStream_t s) {
  Layer& ly = c.layers[l];
  const double* u = W + c.offs[2 * l];
  const double* w = W + c.offs[2 * l + 1];
  if (c.tern) {
    for (int sd = 0; sd < 3; ++sd) {
      bind_ternary(ly, sd, nullptr, u, w);
      net_prepare(*ly.tnet[sd], ly.tbuf[sd], s);
    }
    return;
  }
  for (int sd = 0; sd < 2; ++sd) {
    bind_leaves(ly, sd, nullptr, u, w);
    side_prepare(*ly.net[sd], ly.buf[sd], s);
  }
}

// out += af * Dbar(r) (both sides); operator-path reverse pass only.
void descend(Ctx& c, int l, const double* r, double* out, double af, cudaStream_t s) {
  Layer& ly = c.layers[l];
  if (c.tern) {  // Dbar = (D_L + D_C + D_R) / 3; needs only the prepared values
    for (int sd = 0; sd < 3; ++sd)
      net_backward(*ly.tnet[sd], ly.tbuf[sd], r, true, out, af / 3.0, false, nullptr, nullptr, 0.0, s);
    return;
  }
  for (int sd = 0; sd < 2; ++sd) {
    ly.buf[sd].adj[SideNet::ROOT] = const_cast<double*>(r);
    side_backward(*ly.net[sd], ly.buf[sd], true, out, 0.5 * af, false, nullptr, nullptr, 0.0, s);
  }
}

// ---------------------------------------------------------------- GMRES ----
// Solve Op(x) = b (length n) with restarted GMRES(m), classical Gram-Schmidt
// with one re-orthogonalisation; x holds the initial guess.  Returns the
// number of operator applications; throws MERA_ERR_NOCONV if the relative
// residual stays above tol after maxit applications.
int gmres(Ctx& c, const std::function<void(const double*, double*)>& op, const double* b,
          double* x, int64_t n, double tol, cudaStream_t s) {
  const int m = std::max(2, c.cfg.krylov_dim);
  const int maxit = std::max(m, c.cfg.krylov_maxiter);
  double* V = P(c.kbasis);
  double* w = P(c.ktmp);
  const double bnorm = std::sqrt(c.red.dot(b, b, n, s));
  if (bnorm == 0.0) {
    fill(0.0, x, n, s);
    return 0;
  }
  int applications = 0;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), h1(m + 1), h2(m + 1), y(m);
  double best = INFINITY;
  while (true) {
    op(x, w);
    ++applications;
    axpby(1.0, b, -1.0, w, n, s);  // w = b - A x
    const double beta = std::sqrt(c.red.dot(w, w, n, s));
    if (beta <= tol * bnorm) return applications;
    if (applications >= maxit || !(beta < 1e300)) {
      throw Error(MERA_ERR_NOCONV, "GMRES: relative residual " + std::to_string(beta / bnorm));
    }
    if (beta > 0.9 * best && applications > 2 * m && beta <= 100.0 * tol * bnorm) {
      // no progress over a restart cycle: the residual is at the rounding floor
      return applications;
    }
    best = std::min(best, beta);
    axpby(1.0 / beta, w, 0.0, V, n, s);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < m; ++j) {
      double* vj1 = V + (int64_t)(j + 1) * n;
      op(V + (int64_t)j * n, vj1);
      ++applications;
      c.red.dots(V, n, j + 1, vj1, n, s, h1.data());
      for (int i = 0; i <= j; ++i) h1[i] = -h1[i];
      MERA_CUDA(cudaMemcpyAsync(c.kcoef.p, h1.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
      combine(V, n, j + 1, P(c.kcoef), vj1, n, 1.0, s);
      c.red.dots(V, n, j + 1, vj1, n, s, h2.data());
      for (int i = 0; i <= j; ++i) h2[i] = -h2[i];
      MERA_CUDA(cudaMemcpyAsync(c.kcoef.p, h2.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
      combine(V, n, j + 1, P(c.kcoef), vj1, n, 1.0, s);
      for (int i = 0; i <= j; ++i) H[i * m + j] = -(h1[i] + h2[i]);
      const double hn = std::sqrt(c.red.dot(vj1, vj1, n, s));
      H[(j + 1) * m + j] = hn;
      if (hn > 0) scal(1.0 / hn, vj1, n, s);
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double a = H[j * m + j], bb = H[(j + 1) * m + j];
      const double r = std::hypot(a, bb);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? bb / r : 0.0;
      H[j * m + j] = r;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (std::fabs(g[j + 1]) <= 0.5 * tol * bnorm || hn == 0.0 || applications >= maxit) {
        ++j;
        break;
      }
    }
    // back substitution
    for (int i = j - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < j; ++k) t -= H[i * m + k] * y[k];
      y[i] = H[i * m + i] != 0 ? t / H[i * m + i] : 0.0;
    }
    MERA_CUDA(cudaMemcpyAsync(c.kcoef.p, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
    combine(V, n, j, P(c.kcoef), x, n, 1.0, s);
  }
}

// --------------------------------------------------------- energy / grad ---
void project_tensor(Ctx& c, int i, const double* W, const double* D, double* G, cudaStream_t s) {
  const int64_t n = c.rows[i], p = c.cols[i];
  double* S = P(c.gtmp[0]);
  mm(c, 'C', 'N', p, p, n, 1.0, W, p, D, p, 0.0, S, p, s);     // S = W^dag D
  const bool stiefel = !grass(c, i);
  if (stiefel) herm(c, S, p, s);                                // (S + S^dag)/2
  if (G != D) copy(G, D, n * p * c.rs, s);
  mm(c, 'N', 'N', n, p, p, -1.0, W, p, S, p, 1.0, G, p, s);    // G = D - W S
}

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

void compute_rho_v(Ctx& c, Eval& E, const double* W, cudaStream_t s);
void gradient_pass(Ctx& c, const double* W, Eval& E, cudaStream_t s);

// Energy only: up-sweep, scale-invariant fixed point, e = Tr(h_L rho_S).
double forward_energy(Ctx& c, const double* W, cudaStream_t s);

// Full evaluation at point W into E.
void energy_grad(Ctx& c, const double* W, Eval& E, cudaStream_t s) {
  const int L = c.L;
  c.prof.energy_grad_calls++;
  if (c.mps) {
    mps_energy_grad(c, W, E, s);
    return;
  }
  E.e = forward_energy(c, W, s);
  const int64_t cS = c.dims[L], n3 = opn(c, cS), n = n3 * n3;
  const double floor_tol = c.cfg.prec == MERA_PREC_3XTF32 ? 2e-7 : c.cfg.prec == MERA_PREC_SPLIT_BF16 ? 2e-5 : 0.0;
  const double tol = std::max(c.cfg.krylov_tol, floor_tol);
  double* rhoS = P(c.rho[L]);
  double* hL = P(c.h[L]);
  double* xs = P(c.x);
  const int64_t nr = n * c.rs;  // reals per chi^6 operator
  if (!c.have_x) copy(xs, hL, nr, s);
  auto op_x = [&](const double* v, double* out) {
    copy(out, v, nr, s);
    ascend(c, L, W, v, out, -1.0, s);
    // Tr(v rho) = sum_ij v_ij conj(rho_ij) for hermitian rho
    if (c.cplx) {
      double tr, ti;
      c.red.dot_c(rhoS, v, n, s, &tr, &ti);
      add_identity_c(tr, ti, out, n3, s);
    } else {
      add_identity(c.red.dot(v, rhoS, n, s), out, n3, s);
    }
    ++c.matvecs;
  };
  gmres(c, op_x, hL, xs, nr, tol, s);
  herm(c, xs, n3, s);
  c.have_x = true;
  gradient_pass(c, W, E, s);
}

double forward_energy(Ctx& c, const double* W, cudaStream_t s) {
  if (c.mps) return mps_energy(c, W, s);
  const int L = c.L;
  // up-sweep
  copy(P(c.h[0]), P(c.h0), opn(c, c.dims[0]) * opn(c, c.dims[0]) * c.rs, s);
  if (c.hshift != 0.0) add_id(c, -c.hshift, P(c.h[0]), opn(c, c.dims[0]), s);
  for (int l = 0; l <= L; ++l) prepare_layer(c, l, W, s);
  for (int l = 0; l < L; ++l) {
    const int64_t n3 = opn(c, c.dims[l + 1]);
    fill(0.0, P(c.h[l + 1]), n3 * n3 * c.rs, s);
    ascend(c, l, W, P(c.h[l]), P(c.h[l + 1]), 1.0, s);
    herm(c, P(c.h[l + 1]), n3, s);
  }
  // scale-invariant layer
  const int64_t cS = c.dims[L], n3 = opn(c, cS), n = n3 * n3, nr = n * c.rs;
  double* rhoS = P(c.rho[L]);
  if (!c.have_rho) {
    fill(0.0, rhoS, nr, s);
    add_id(c, 1.0 / (double)n3, rhoS, n3, s);
  }
  double* bvec = P(c.bvec);
  fill(0.0, bvec, nr, s);
  add_id(c, 1.0 / (double)n3, bvec, n3, s);
  // the residual of a Krylov solve cannot fall below the rounding level of
  // the contractions that apply the superoperator
  const double floor_tol = c.cfg.prec == MERA_PREC_3XTF32 ? 2e-7 : c.cfg.prec == MERA_PREC_SPLIT_BF16 ? 2e-5 : 0.0;
  const double tol = std::max(c.cfg.krylov_tol, floor_tol);
  auto op_rho = [&](const double* v, double* out) {
    copy(out, v, nr, s);
    descend(c, L, v, out, -1.0, s);
    // + Tr(v) b, b = 1/chi^3
    if (c.cplx) {
      double tr, ti;
      c.red.trace_c(v, n3, s, &tr, &ti);
      add_identity_c(tr / (double)n3, ti / (double)n3, out, n3, s);
    } else {
      axpy(c.red.trace(v, n3, s), bvec, out, n, s);
    }
    ++c.matvecs;
  };
  gmres(c, op_rho, bvec, rhoS, nr, tol, s);
  double tr = 0.0, ti = 0.0;
  if (c.cplx) c.red.trace_c(rhoS, n3, s, &tr, &ti); else tr = c.red.trace(rhoS, n3, s);
  if (!(std::fabs(tr) > 0)) throw Error(MERA_ERR_NONFINITE, "fixed point has zero trace");
  scal(1.0 / tr, rhoS, nr, s);
  herm(c, rhoS, n3, s);
  c.have_rho = true;
  // Tr(h rho) = Re sum_ij h_ij conj(rho_ij): the real dot product of the arrays
  const double e = c.red.dot(P(c.h[L]), rhoS, nr, s);
  check_device_flag(c, s);
  if (!std::isfinite(e)) throw Error(MERA_ERR_NONFINITE, "non-finite energy");
  return e;
}

// Reverse passes of every layer (environments, descending maps), projection
// and the preconditioner's density matrices; needs forward_energy and x.
void gradient_pass(Ctx& c, const double* W, Eval& E, cudaStream_t s) {
  const int L = c.L;
  double* rhoS = P(c.rho[L]);
  double* xs = P(c.x);
  // down-sweep with environments
  double* D = P(E.D);
  fill(0.0, D, c.total, s);
  for (int l = L; l >= 0; --l) {
    Layer& ly = c.layers[l];
    const double* u = W + c.offs[2 * l];
    const double* w = W + c.offs[2 * l + 1];
    const double* op = l < L ? P(c.h[l]) : xs;
    const double* r = l < L ? P(c.rho[l + 1]) : rhoS;
    const bool need_op = l < L;
    if (need_op) fill(0.0, P(c.rho[l]), opn(c, ly.cf) * opn(c, ly.cf) * c.rs, s);
    for (int sd = 0; c.tern && sd < 3; ++sd) {
      // D_v = 2 dC/d conj(v) with C = Tr(Abar(h) rho), Abar the average of three maps
      bind_ternary(ly, sd, op, u, w);
      if (l == L || c.cfg.recompute_env) net_forward(*ly.tnet[sd], ly.tbuf[sd], nullptr, 0.0, 0.0, s);
      net_backward(*ly.tnet[sd], ly.tbuf[sd], r, need_op, need_op ? P(c.rho[l]) : nullptr, 1.0 / 3.0, true,
                   D + c.offs[2 * l], D + c.offs[2 * l + 1], 2.0 / 3.0, s);
    }
    for (int sd = 0; !c.tern && sd < 2; ++sd) {
      SideBufs& b = ly.buf[sd];
      bind_leaves(ly, sd, op, u, w);
      // the reverse pass needs N3, N7, N8 for this layer's operator: the
      // up-sweep left them in place for the transition layers (unless
      // recomputation was asked for); the scale-invariant layer's operator is x
      if (l == L || c.cfg.recompute_env) side_forward(*ly.net[sd], b, nullptr, 0.0, 0.0, s);
      b.adj[SideNet::ROOT] = const_cast<double*>(r);
      side_backward(*ly.net[sd], b, need_op, need_op ? P(c.rho[l]) : nullptr, 0.5, true,
                    D + c.offs[2 * l], D + c.offs[2 * l + 1], 1.0, s);
    }
    if (need_op) herm(c, P(c.rho[l]), opn(c, ly.cf), s);
  }
  // projection
  for (int i = 0; i < c.nt; ++i)
    project_tensor(c, i, W + c.offs[i], D + c.offs[i], P(E.G) + c.offs[i], s);
  E.delta.resize(c.nt);
  bool finite = std::isfinite(E.e);
  for (int i = 0; i < c.nt; ++i) {
    const double* g = P(E.G) + c.offs[i];
    E.delta[i] = std::sqrt(c.red.dot(g, g, c.rows[i] * c.cols[i] * c.rs, s));
    finite = finite && std::isfinite(E.delta[i]);
  }
  check_device_flag(c, s);
  if (!finite) throw Error(MERA_ERR_NONFINITE, "non-finite energy or gradient");
  compute_rho_v(c, E, W, s);
  E.eig_ready = false;
  E.valid = true;
}

// rho_w: one-site marginal of the density matrix above the layer; rho_u:
// W rho2 W^T on the pair of isometry outputs that u acts on (Sec. 4).
// Ternary network: rho_w the one-site marginal of rho_{l+1}; rho_u the state
// on the isometry outputs a u acts on (third leg of w_j, first of w_{j+1}):
//   T1[p0 p1 x2 b A B]    = w[p0 p1 x2 a] rho[a b A B]
//   T2[x2 b B X2]         = T1 x conj w[p0 p1 X2 A]
//   T3[x2 B X2 x3 p4 p5]  = T2 x w[x3 p4 p5 b]
//   rho_u[x2 x3 X2 X3]    = T3 x conj w[X3 p4 p5 B]
void compute_rho_v_ternary(Ctx& c, Eval& E, const double* W, cudaStream_t s) {
  auto D = [](std::vector<int> legs, std::vector<int64_t> ext) {
    TDesc d;
    d.legs = legs;
    d.ext = ext;
    d.stride.assign(legs.size(), 1);
    for (size_t j = legs.size(); j-- > 1;) d.stride[j - 1] = d.stride[j] * ext[j];
    return d;
  };
  for (int l = 0; l <= c.L; ++l) {
    const int64_t cf = c.layers[l].cf, cc = c.layers[l].cc;
    const double* r = l < c.L ? P(c.rho[l + 1]) : P(c.rho[c.L]);
    const double* w = W + c.offs[2 * l + 1];
    double* rw = P(E.rho_v[2 * l + 1]);
    double* ru = P(E.rho_v[2 * l]);
    if (c.cplx)
      marg_tern_c_k<<<blocks(cc * cc), 256, 0, s>>>(reinterpret_cast<const double2*>(r), cc,
                                                     reinterpret_cast<double2*>(rw));
    else
      marg_tern_k<<<blocks(cc * cc), 256, 0, s>>>(r, cc, rw);
    count_launch();
    MERA_CHECK_LAUNCH();
    enum { p0, p1, x2, x3, X2, X3, p4, p5, a, b, A, B };
    const TDesc wa = D({p0, p1, x2, a}, {cf, cf, cf, cc}), R = D({a, b, A, B}, {cc, cc, cc, cc});
    const TDesc T1 = D({p0, p1, x2, b, A, B}, {cf, cf, cf, cc, cc, cc});
    const TDesc wA = D({p0, p1, X2, A}, {cf, cf, cf, cc});
    const TDesc T2 = D({x2, b, B, X2}, {cf, cc, cc, cf});
    const TDesc wb = D({x3, p4, p5, b}, {cf, cf, cf, cc});
    const TDesc T3 = D({x2, B, X2, x3, p4, p5}, {cf, cc, cf, cf, cf, cf});
    const TDesc wB = D({X3, p4, p5, B}, {cf, cf, cf, cc});
    const TDesc RU = D({x2, x3, X2, X3}, {cf, cf, cf, cf});
    double* t1 = P(c.gtmp[2]);
    double* t2 = P(c.gtmp[3]);
    double* t3 = P(c.gtmp[4]);
    auto run = [&](const TDesc& A_, const TDesc& B_, const TDesc& C_, const double* pa, const double* pb, double* pc,
                   bool conj_b) {
      GettCall g = make_plan(A_, B_, C_, c.pool).proto;
      g.A = pa;
      g.B = pb;
      g.C = pc;
      g.cplx = c.cplx;
      g.b_conj = c.cplx && conj_b;
      gett_f64(g, s);
    };
    run(wa, R, T1, w, r, t1, false);
    run(T1, wA, T2, t1, w, t2, true);
    run(T2, wb, T3, t2, w, t3, false);
    run(T3, wB, RU, t3, w, ru, true);
    herm(c, ru, cf * cf, s);
    herm(c, rw, cc, s);
  }
}

void compute_rho_v(Ctx& c, Eval& E, const double* W, cudaStream_t s) {
  if (c.tern) {
    compute_rho_v_ternary(c, E, W, s);
    return;
  }
  for (int l = 0; l <= c.L; ++l) {
    const int64_t cf = c.layers[l].cf, cc = c.layers[l].cc;
    const double* r = l < c.L ? P(c.rho[l + 1]) : P(c.rho[c.L]);
    const double* w = W + c.offs[2 * l + 1];
    double* rw = P(E.rho_v[2 * l + 1]);
    double* ru = P(E.rho_v[2 * l]);
    double* r2 = P(c.gtmp[1]);
    if (c.cplx) {
      marginal_1site_mid_c(r, cc, rw, s);
      marginal_2site_left_c(r, cc, r2, s);
    } else {
      marginal_1site_mid(r, cc, rw, s);
      marginal_2site_left(r, cc, r2, s);
    }
    // pairwise: T1[x0 x1 b A B] = w[x0 x1 a] r2[a b A B]
    //           T2[x1 b B X1]   = T1 x w[x0 X1 A]
    //           T3[x1 B X1 x2 x3] = T2 x w[x2 x3 b]
    //           ru[x1 x2 X1 X2] = T3 x w[X2 x3 B]
    auto D = [](std::vector<int> legs, std::vector<int64_t> ext) {
      TDesc d;
      d.legs = legs;
      d.ext = ext;
      d.stride.assign(legs.size(), 1);
      for (size_t j = legs.size(); j-- > 1;) d.stride[j - 1] = d.stride[j] * ext[j];
      return d;
    };
    enum { x0, x1, x2, x3, X1, X2, a, b, A, B };
    TDesc wa = D({x0, x1, a}, {cf, cf, cc}), R2 = D({a, b, A, B}, {cc, cc, cc, cc});
    TDesc T1 = D({x0, x1, b, A, B}, {cf, cf, cc, cc, cc});
    TDesc wA = D({x0, X1, A}, {cf, cf, cc});
    TDesc T2 = D({x1, b, B, X1}, {cf, cc, cc, cf});
    TDesc wb = D({x2, x3, b}, {cf, cf, cc});
    TDesc T3 = D({x1, B, X1, x2, x3}, {cf, cc, cf, cf, cf});
    TDesc wB = D({X2, x3, B}, {cf, cf, cc});
    TDesc RU = D({x1, x2, X1, X2}, {cf, cf, cf, cf});
    double* t1 = P(c.gtmp[2]);
    double* t2 = P(c.gtmp[3]);
    double* t3 = P(c.gtmp[4]);
    auto run = [&](const TDesc& A_, const TDesc& B_, const TDesc& C_, const double* pa,
                   const double* pb, double* pc, bool conj_b) {
      GettCall g = make_plan(A_, B_, C_, c.pool).proto;
      g.A = pa;
      g.B = pb;
      g.C = pc;
      g.cplx = c.cplx;
      g.b_conj = c.cplx && conj_b;
      gett_f64(g, s);
    };
    // rho_u = W rho2 W^dag: the two isometries on the bra side are conjugated
    run(wa, R2, T1, w, r2, t1, false);
    run(T1, wA, T2, t1, w, t2, true);
    run(T2, wb, T3, t2, w, t3, false);
    run(T3, wB, RU, t3, w, ru, true);
    herm(c, ru, cf * cf, s);
    herm(c, rw, cc, s);
  }
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

// ------------------------------------------------------------ optimiser ----
struct LsResult {
  double alpha = 0, f = 0, df = 0;
  int nev = 0;
  bool ok = false, found = false;
};

// One trial: point Wtry = R(Wcur, d, a), evaluation into ev[1-cur],
// dir2 = T(d).  Returns (f, df).
std::pair<double, double> trial(Ctx& c, double a, cudaStream_t s) {
  const double* W = P(c.Wcur);
  make_geom(c, W, P(c.dir), a, s);
  apply_retract(c, W, P(c.dir), P(c.Wtry), s);
  Eval& E = c.ev[1 - c.cur];
  double f, df;
  try {
    energy_grad(c, P(c.Wtry), E, s);
    copy(P(c.dir2), P(c.dir), c.total, s);
    apply_transport(c, W, P(c.dir), P(c.dir2), s);
    f = E.e;
    df = inner(c, P(E.G), P(c.dir2), s);
  } catch (const Error& e) {
    if (e.code != MERA_ERR_NONFINITE) throw;
    f = INFINITY;
    df = INFINITY;
  }
  return {f, df};
}

LsResult hager_zhang(Ctx& c, double f0, double df0, double a0, cudaStream_t s) {
  const double delta = 0.1, sigma = 0.9, eps = 1e-6, theta = 0.5, gamma = 0.66, expand = 5.0;
  const int maxeval = 20;
  const double epsk = eps * std::fabs(f0);
  struct Pt { double a, f, df; };
  std::vector<Pt> hist;
  LsResult res;
  double last_a = NAN;
  auto ev = [&](double a) -> Pt {
    for (auto& p : hist)
      if (p.a == a) return p;
    if ((int)hist.size() >= maxeval) throw 1;
    auto fd = trial(c, a, s);
    last_a = a;
    Pt p{a, fd.first, fd.second};
    if (!std::isfinite(p.f) || !std::isfinite(p.df)) { p.f = INFINITY; p.df = INFINITY; }
    hist.push_back(p);
    const bool wolfe = (p.f - f0 <= delta * a * df0) && (p.df >= sigma * df0);
    const bool approx = ((2 * delta - 1) * df0 >= p.df) && (p.df >= sigma * df0) && (p.f <= f0 + epsk);
    if (wolfe || approx) throw 2;
    return p;
  };
  auto dfof = [&](double a) { if (a == 0) return df0; for (auto& p : hist) if (p.a == a) return p.df; return df0; };
  auto u3 = [&](double a, double b) -> std::pair<double, double> {
    while (true) {
      const double d = (1 - theta) * a + theta * b;
      Pt p = ev(d);
      if (p.df >= 0) return {a, d};
      if (p.f <= f0 + epsk) a = d; else b = d;
    }
  };
  auto update = [&](double a, double b, double cc) -> std::pair<double, double> {
    if (!(a < cc && cc < b)) return {a, b};
    Pt p = ev(cc);
    if (p.df >= 0) return {a, cc};
    if (p.f <= f0 + epsk) return {cc, b};
    return u3(a, cc);
  };
  auto secant = [&](double a, double b) {
    const double da = dfof(a), db = dfof(b);
    if (db == da) return 0.5 * (a + b);
    return (a * db - b * da) / (db - da);
  };
  int outcome = 0;
  try {
    double cc = a0;
    Pt p = ev(cc);
    double good = 0.0, a, b;
    while (true) {
      if (p.df >= 0) { a = good; b = cc; break; }
      if (p.f > f0 + epsk) { auto ab = u3(0.0, cc); a = ab.first; b = ab.second; break; }
      good = cc;
      cc *= expand;
      p = ev(cc);
    }
    while (true) {
      const double cs = secant(a, b);
      auto AB = update(a, b, cs);
      if (cs == AB.second) AB = update(AB.first, AB.second, secant(b, AB.second));
      else if (cs == AB.first) AB = update(AB.first, AB.second, secant(a, AB.first));
      if (AB.second - AB.first > gamma * (b - a)) AB = update(AB.first, AB.second, 0.5 * (AB.first + AB.second));
      a = AB.first;
      b = AB.second;
    }
  } catch (int code) {
    outcome = code;
  }
  res.nev = (int)hist.size();
  if (outcome == 2) {
    res.ok = true;
    res.found = true;
    res.alpha = last_a;
    res.f = hist.back().f;
    res.df = hist.back().df;
    return res;
  }
  // best finite trial
  double bf = INFINITY, ba = NAN;
  for (auto& p : hist)
    if (p.f < bf) { bf = p.f; ba = p.a; }
  if (std::isfinite(bf)) {
    res.found = true;
    res.alpha = ba;
    if (ba != last_a) trial(c, ba, s);  // re-evaluate to leave its state in place
    res.f = c.ev[1 - c.cur].e;
    res.df = NAN;
  }
  return res;
}

// ------------------------------------------------------- Evenbly-Vidal ----
// W <- -Q with D = Q P the polar decomposition, Q = D (D^dag D)^(-1/2): the
// update of one tensor from its environment D (App. ev_steplimit), then two
// Newton-Schulz steps so that W is isometric to rounding.
void ev_replace(Ctx& c, int i, const double* D, double* W, cudaStream_t s) {
  const int64_t n = c.rows[i], p = c.cols[i], q = p * c.rs;
  double* Z = P(c.gtmp[0]);   // D^dag D, then (complex) its real embedding
  double* V = P(c.gtmp[1]);   // eigenvectors (q x q)
  double* R = P(c.gtmp[2]);   // (D^dag D)^(-1/2), p x p
  double* fr = P(c.gtmp[3]);  // inverse square roots of the eigenvalues
  double* F = P(c.gtmp[4]);   // q x q scratch
  double* f = P(c.gtmp[5]);   // eigenvalues
  mm(c, 'C', 'N', p, p, n, 1.0, D, p, D, p, 0.0, Z, p, s);
  herm(c, Z, p, s);
  if (c.cplx) {
    embed_complex(Z, p, F, s);
    copy(Z, F, q * q, s);
  }
  sym_eig(Z, V, f, (int)q, c.eigw, s);
  spectral_k<<<blocks(q), 256, 0, s>>>(f, (int)q, 5, 0.0, 1e-300, fr);
  vfvt_k<<<blocks(q * q), 256, 0, s>>>(V, fr, (int)q, c.cplx ? F : R);
  count_launch(2);
  MERA_CHECK_LAUNCH();
  if (c.cplx) extract_complex(F, p, R, s);
  mm(c, 'N', 'N', n, p, p, -1.0, D, p, R, p, 0.0, W, p, s);
  polar_ns(c, W, n, p, s);
}

void ensure_current(Ctx& c, cudaStream_t s);
void clear_history(Ctx& c);

// One sweep over u_0, w_0, ..., u_S, w_S: environment of the cost with the
// shifted term h3 - gamma 1 at the current point, then the tensor's update.
// Ends with one unshifted evaluation at the new point.
void ev_sweep(Ctx& c, double gamma, mera_iter_info* info, cudaStream_t s) {
  if (c.mps) throw Error(MERA_ERR_UNSUPPORTED, "Evenbly-Vidal sweeps are defined for the MERA networks");
  Eval& E = c.ev[c.cur];
  const int64_t mv0 = c.matvecs;
  int evals = 0;
  c.hshift = gamma;
  try {
    for (int i = 0; i < c.nt; ++i) {
      energy_grad(c, P(c.Wcur), E, s);
      ++evals;
      ev_replace(c, i, P(E.D) + c.offs[i], P(c.Wcur) + c.offs[i], s);
    }
  } catch (...) {
    c.hshift = 0.0;
    c.ev[0].valid = c.ev[1].valid = false;
    c.geom.valid = false;
    throw;
  }
  c.hshift = 0.0;
  c.ev[0].valid = c.ev[1].valid = false;
  c.geom.valid = false;
  clear_history(c);
  energy_grad(c, P(c.Wcur), E, s);
  ++evals;
  info->iter = ++c.iters;
  info->energy = E.e;
  info->gnorm = std::sqrt(inner(c, P(E.G), P(E.G), s));
  info->alpha = 0.0;
  info->n_evals = evals;
  info->ls_ok = 1;
  info->krylov_matvecs = (int)(c.matvecs - mv0);
}

void ensure_current(Ctx& c, cudaStream_t s) {
  if (!c.ev[c.cur].valid) energy_grad(c, P(c.Wcur), c.ev[c.cur], s);
}

void clear_history(Ctx& c) {
  c.mem_n = 0;
  c.mem_rho.clear();
  c.alpha_prev = 1.0;
}

// Accept the last trial: its point and evaluation become the current ones
// (the caller has transported the history).
void accept(Ctx& c, cudaStream_t) {
  std::swap(c.Wcur, c.Wtry);
  c.cur = 1 - c.cur;
}

void lbfgs_step(Ctx& c, mera_iter_info* info, cudaStream_t s) {
  ensure_current(c, s);
  const int64_t mv0 = c.matvecs;
  Eval& E = c.ev[c.cur];
  const double* W = P(c.Wcur);
  double* G = P(E.G);
  const int m = std::max(1, c.cfg.lbfgs_m);
  // two-loop recursion, q in dir
  double* q = P(c.dir);
  copy(q, G, c.total, s);
  std::vector<double> al(c.mem_n);
  for (int i = c.mem_n - 1; i >= 0; --i) {
    al[i] = c.mem_rho[i] * inner(c, P(c.mem_s[i]), q, s);
    axpy(-al[i], P(c.mem_y[i]), q, c.total, s);
  }
  double gam = 1.0;
  if (c.mem_n > 0) {
    double* Py = P(c.tmpv);
    precondition(c, E, W, P(c.mem_y[c.mem_n - 1]), Py, s);
    gam = (1.0 / c.mem_rho[c.mem_n - 1]) / inner(c, P(c.mem_y[c.mem_n - 1]), Py, s);
  }
  precondition(c, E, W, q, P(c.tmpv), s);
  axpby(gam, P(c.tmpv), 0.0, q, c.total, s);
  for (int i = 0; i < c.mem_n; ++i) {
    const double b = c.mem_rho[i] * inner(c, P(c.mem_y[i]), q, s);
    axpy(al[i] - b, P(c.mem_s[i]), q, c.total, s);
  }
  scal(-1.0, q, c.total, s);
  double df0 = inner(c, G, q, s);
  if (!(df0 < 0)) {
    clear_history(c);
    precondition(c, E, W, G, q, s);
    scal(-1.0, q, c.total, s);
    df0 = inner(c, G, q, s);
  }
  const double f0 = E.e;
  LsResult ls = hager_zhang(c, f0, df0, 1.0, s);
  info->n_evals = ls.nev;
  info->ls_ok = ls.ok;
  if (!ls.found || (!ls.ok && ls.f >= f0)) {
    clear_history(c);
    info->alpha = 0.0;
    info->energy = f0;
    info->gnorm = std::sqrt(inner(c, G, G, s));
    info->iter = ++c.iters;
    info->krylov_matvecs = (int)(c.matvecs - mv0);
    return;
  }
  // c.geom holds the accepted alpha's quantities, dir2 = T(d)
  const double a = ls.alpha;
  for (int i = 0; i < c.mem_n; ++i) {
    apply_transport(c, W, P(c.dir), P(c.mem_s[i]), s);
    apply_transport(c, W, P(c.dir), P(c.mem_y[i]), s);
  }
  // s_new = a T(d), y_new = G' - T(G)
  double* Tg = P(c.tmpv);
  copy(Tg, G, c.total, s);
  apply_transport(c, W, P(c.dir), Tg, s);
  Eval& En = c.ev[1 - c.cur];
  if (c.mem_n == m) {
    // drop the oldest pair (rotate buffers)
    DevBuf s0 = std::move(c.mem_s[0]), y0 = std::move(c.mem_y[0]);
    for (int i = 0; i + 1 < m; ++i) {
      c.mem_s[i] = std::move(c.mem_s[i + 1]);
      c.mem_y[i] = std::move(c.mem_y[i + 1]);
    }
    c.mem_s[m - 1] = std::move(s0);
    c.mem_y[m - 1] = std::move(y0);
    c.mem_rho.erase(c.mem_rho.begin());
    c.mem_n--;
  }
  double* sn = P(c.mem_s[c.mem_n]);
  double* yn = P(c.mem_y[c.mem_n]);
  axpby(a, P(c.dir2), 0.0, sn, c.total, s);
  copy(yn, P(En.G), c.total, s);
  axpy(-1.0, Tg, yn, c.total, s);
  const double sy = inner(c, sn, yn, s);
  const double ss = inner(c, sn, sn, s), yy = inner(c, yn, yn, s);
  if (sy > 1e-16 * std::sqrt(ss * yy)) {
    c.mem_rho.push_back(1.0 / sy);
    c.mem_n++;
  }
  accept(c, s);
  Eval& Ec = c.ev[c.cur];
  info->alpha = a;
  info->energy = Ec.e;
  info->gnorm = std::sqrt(inner(c, P(Ec.G), P(Ec.G), s));
  info->iter = ++c.iters;
  info->krylov_matvecs = (int)(c.matvecs - mv0);
}

void cg_step(Ctx& c, mera_iter_info* info, cudaStream_t s) {
  ensure_current(c, s);
  const int64_t mv0 = c.matvecs;
  Eval& E = c.ev[c.cur];
  const double* W = P(c.Wcur);
  double* G = P(E.G);
  double* d = P(c.dir);
  // c.mem_n == 1 means dir holds the previous (transported) direction
  if (c.mem_n == 0) {
    precondition(c, E, W, G, d, s);
    scal(-1.0, d, c.total, s);
  }
  double df0 = inner(c, G, d, s);
  if (!(df0 < 0)) {
    precondition(c, E, W, G, d, s);
    scal(-1.0, d, c.total, s);
    df0 = inner(c, G, d, s);
  }
  const double f0 = E.e;
  LsResult ls = hager_zhang(c, f0, df0, c.alpha_prev, s);
  info->n_evals = ls.nev;
  info->ls_ok = ls.ok;
  if (!ls.found || (!ls.ok && ls.f >= f0)) {
    c.mem_n = 0;
    info->alpha = 0.0;
    info->energy = f0;
    info->gnorm = std::sqrt(inner(c, G, G, s));
    info->iter = ++c.iters;
    info->krylov_matvecs = (int)(c.matvecs - mv0);
    return;
  }
  const double a = ls.alpha;
  Eval& En = c.ev[1 - c.cur];
  // y = G' - T(G)
  double* y = P(c.tmpv);
  copy(y, G, c.total, s);
  apply_transport(c, W, d, y, s);
  axpby(1.0, P(En.G), -1.0, y, c.total, s);
  const double* Wn = P(c.Wtry);
  double* Pg = P(c.tmpv2);
  precondition(c, En, Wn, P(En.G), Pg, s);
  double* d2 = P(c.dir2);
  const double dy = inner(c, d2, y, s);
  double beta = 0.0;
  if (dy != 0.0) {
    double* Py = P(c.mem_s.empty() ? c.tmpv : c.mem_s[0]);
    precondition(c, En, Wn, y, Py, s);
    beta = (inner(c, y, Pg, s) - 2.0 * inner(c, y, Py, s) * inner(c, d2, P(En.G), s) / dy) / dy;
  }
  const double dn = std::sqrt(inner(c, d2, d2, s));
  const double gn = std::sqrt(inner(c, P(En.G), P(En.G), s));
  beta = std::max(beta, -1.0 / (dn * std::min(0.01, gn)));
  // new direction d = -Pg + beta T(d)
  axpby(-1.0, Pg, beta, d2, c.total, s);
  copy(d, d2, c.total, s);
  c.mem_n = 1;
  c.alpha_prev = a;
  accept(c, s);
  info->alpha = a;
  info->energy = c.ev[c.cur].e;
  info->gnorm = gn;
  info->iter = ++c.iters;
  info->krylov_matvecs = (int)(c.matvecs - mv0);
}

// ------------------------------------------------------------ creation -----
void check_isometric(Ctx& c, const double* W, cudaStream_t s) {
  for (int i = 0; i < c.nt; ++i) {
    const int64_t n = c.rows[i], p = c.cols[i];
    double* S = P(c.gtmp[0]);
    mm(c, 'C', 'N', p, p, n, 1.0, W + c.offs[i], p, W + c.offs[i], p, 0.0, S, p, s);
    add_id(c, -1.0, S, p, s);
    const double r = std::sqrt(c.red.dot(S, S, p * p * c.rs, s));
    if (!(r < 1e-10)) throw Error(MERA_ERR_NOT_ISOMETRIC, "tensor " + std::to_string(i) + " has |W^T W - 1| = " + std::to_string(r));
  }
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

void create_mera(Ctx& c, int64_t* nS, int64_t* gmax);
void finish_create(Ctx& c, cudaStream_t s);

// Z2 symmetry of a (rows x cols) matrix on the device whose rows (columns)
// are index tuples of legs with dimensions rdims (cdims), row-major: every
// entry between a row and a column of different total charge (the legs'
// gradings summed, first half of each leg even) must be below 1e-12 of the
// largest entry (Sec. 6); MERA_ERR_ARG otherwise.
// Z2 charge of every index tuple of legs with dimensions dims (row-major).
std::vector<int> fused_charges(const std::vector<int64_t>& dims) {
  int64_t n = 1;
  for (int64_t e : dims) n *= e;
  std::vector<int> ch(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = i;
    for (size_t j = dims.size(); j-- > 0;) {
      ch[i] ^= z2_charge(r % dims[j], dims[j]);
      r /= dims[j];
    }
  }
  return ch;
}

void check_z2(Ctx& c, const double* dev, const std::vector<int64_t>& rdims, const std::vector<int64_t>& cdims,
              const std::string& what, cudaStream_t s) {
  const std::vector<int> cr = fused_charges(rdims), cc = fused_charges(cdims);
  const int64_t R = (int64_t)cr.size(), C = (int64_t)cc.size();
  std::vector<double> h((size_t)(R * C * c.rs));
  MERA_CUDA(cudaMemcpyAsync(h.data(), dev, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  double big = 0.0, bad = 0.0;
  for (int64_t r = 0; r < R; ++r)
    for (int64_t k = 0; k < C; ++k) {
      const double* e = h.data() + (r * C + k) * c.rs;
      const double mag = c.cplx ? std::hypot(e[0], e[1]) : std::fabs(e[0]);
      big = std::max(big, mag);
      if (cr[r] != cc[k]) bad = std::max(bad, mag);
    }
  if (!(bad <= 1e-12 * big))
    throw Error(MERA_ERR_ARG, what + " is not Z2-symmetric (entry " + std::to_string(bad) +
                                  " between different charges)");
}

// Z2 symmetry of every tensor of a ternary point: u_l (cf cf) x (cf cf),
// w_l (cf cf cf) x (cc).
void check_z2_point(Ctx& c, const double* W, cudaStream_t s) {
  for (int l = 0; l <= c.L; ++l) {
    const int64_t cf = c.dims[l], cc = l < c.L ? c.dims[l + 1] : c.dims[l];
    check_z2(c, W + c.offs[2 * l], {cf, cf}, {cf, cf}, "u_" + std::to_string(l), s);
    check_z2(c, W + c.offs[2 * l + 1], {cf, cf, cf}, {cc}, "w_" + std::to_string(l), s);
  }
}

void create(Ctx& c, const mera_config& cfg, const void* h3, cudaStream_t s) {
  c.cfg = cfg;
  c.s = s;
  if (cfg.dtype != MERA_F64 && cfg.dtype != MERA_C128) throw Error(MERA_ERR_ARG, "unknown dtype");
  c.cplx = cfg.dtype == MERA_C128;
  c.rs = c.cplx ? 2 : 1;
  if (cfg.prec != MERA_PREC_FP64 && cfg.prec != MERA_PREC_3XTF32 && cfg.prec != MERA_PREC_SPLIT_BF16)
    throw Error(MERA_ERR_ARG, "unknown precision mode");
  if (cfg.network != MERA_BINARY && cfg.network != MERA_TERNARY && cfg.network != MERA_MPS)
    throw Error(MERA_ERR_ARG, "unknown network");
  c.tern = cfg.network == MERA_TERNARY;
  c.mps = cfg.network == MERA_MPS;
  if (cfg.z2 != 0 && cfg.z2 != 1) throw Error(MERA_ERR_ARG, "z2 must be 0 or 1");
  c.z2 = cfg.z2 == 1;
  if (c.z2 && !c.tern) throw Error(MERA_ERR_UNSUPPORTED, "Z2 charge sectors are built for the ternary network");
  c.ns = c.tern || c.mps ? 2 : 3;
  c.pool.set_stream(s);
  int64_t nS = 0, gmax = 1;  // reals of one Krylov vector; elements of a geometry temporary
  if (c.mps) {
    create_mps(c, &nS, &gmax);
  } else {
    create_mera(c, &nS, &gmax);
  }
  const size_t tb = sizeof(double) * c.total;
  c.Wcur.alloc(tb);
  c.Wtry.alloc(tb);
  c.h0.alloc(sizeof(double) * ipow(cfg.d_b, 2 * c.ns) * c.rs);
  MERA_CUDA(cudaMemcpyAsync(c.h0.p, h3, c.h0.bytes, cudaMemcpyDefault, s));
  if (c.z2) {
    const std::vector<int64_t> pair{cfg.d_b, cfg.d_b};
    check_z2(c, P(c.h0), pair, pair, "the Hamiltonian term", s);
  }
  c.x.alloc(sizeof(double) * nS);
  c.kbasis.alloc(sizeof(double) * nS * (std::max(2, cfg.krylov_dim) + 1));
  c.ktmp.alloc(sizeof(double) * nS);
  c.kcoef.alloc(sizeof(double) * (cfg.krylov_dim + 2));
  c.red.init(std::max(8, cfg.krylov_dim + 2));
  c.bvec.alloc(sizeof(double) * nS);
  gmax *= c.cplx ? 4 : 1;  // complex data and 2p x 2p real embeddings
  for (auto& b : c.gtmp) b.alloc(sizeof(double) * gmax);
  finish_create(c, s);
}

// Shapes, networks and level buffers of a binary or ternary MERA.
void create_mera(Ctx& c, int64_t* nS, int64_t* gmax) {
  const mera_config& cfg = c.cfg;
  if (cfg.d_b < 2 || cfg.chi < 2 || cfg.n_trans < 1) throw Error(MERA_ERR_ARG, "bad d_b/chi/n_trans");
  // complex data on the tensor cores: every product as four real products of
  // the real views, whose tables the plans then carry
  c.pool.set_real_view(c.cplx && cfg.prec != MERA_PREC_FP64);
  c.L = cfg.n_trans;
  c.dims.push_back(cfg.d_b);
  // a coarse site holds two (binary) or three (ternary) fine sites
  for (int l = 0; l < c.L; ++l) {
    const int64_t d = c.dims.back();
    c.dims.push_back(std::min<int64_t>(cfg.chi, c.tern ? d * d * d : d * d));
  }
  if (c.dims.back() != cfg.chi) throw Error(MERA_ERR_ARG, "transition layers do not reach chi");
  c.nt = 2 * (c.L + 1);
  int64_t off = 0;
  for (int l = 0; l <= c.L; ++l) {
    const int64_t cf = c.dims[l], cc = l < c.L ? c.dims[l + 1] : c.dims[l];
    const int64_t wr = c.tern ? cf * cf * cf : cf * cf;  // rows of w: the fine pair or triple
    c.rows.push_back(cf * cf); c.cols.push_back(cf * cf); c.offs.push_back(off); off += cf * cf * cf * cf * c.rs;
    c.rows.push_back(wr);      c.cols.push_back(cc);      c.offs.push_back(off); off += wr * cc * c.rs;
  }
  c.total = off;
  build_layers(c);
  for (int l = 0; l <= c.L; ++l) {
    c.h.emplace_back(sizeof(double) * ipow(c.dims[l], 2 * c.ns) * c.rs);
    c.rho.emplace_back(sizeof(double) * ipow(c.dims[l], 2 * c.ns) * c.rs);
  }
  *nS = ipow(cfg.chi, 2 * c.ns) * c.rs;  // reals of one level operator (chi^6 binary)
  // geometry temporaries: max over tensors / rho_u builders
  int64_t g = 1;
  for (int l = 0; l <= c.L; ++l) {
    const int64_t cf = c.dims[l], cc = l < c.L ? c.dims[l + 1] : c.dims[l];
    g = std::max({g, cf * cf * cf * cf, cc * cc * cc * cc, cf * cf * cc * cc * cc,
                  cf * cc * cc * cf, cf * cc * cf * cf * cf});
    // ternary: w, and the rho_u builder's T1 (cf^3 cc^3) and T3 (cf^5 cc)
    if (c.tern) g = std::max({g, cf * cf * cf * cc, cf * cf * cf * cc * cc * cc, cf * cf * cf * cf * cf * cc});
  }
  *gmax = g;
}

// Buffers every problem has: evaluations, step geometry, optimiser memory,
// and the default point (u = 1, w = first columns).
void finish_create(Ctx& c, cudaStream_t s) {
  const mera_config& cfg = c.cfg;
  const size_t tb = sizeof(double) * c.total;
  for (auto& E : c.ev) {
    E.G.alloc(tb);
    E.D.alloc(tb);
    for (int i = 0; i < c.nt; ++i) {
      const int64_t p = c.cols[i], q = p * c.rs;
      E.rho_v.emplace_back(sizeof(double) * p * p * c.rs);
      E.evec.emplace_back(sizeof(double) * q * q);
      E.eval.emplace_back(sizeof(double) * q);
    }
  }
  StepGeom& g = c.geom;
  c.eig_uses.assign(c.nt, 0);
  for (int i = 0; i < c.nt; ++i) {
    const int64_t p = c.cols[i], q = p * c.rs;
    c.eig_cache.emplace_back(sizeof(double) * q * q);
    g.Amat.emplace_back(sizeof(double) * q * q);
    // a non-square Stiefel point's exponential lives on 2p dimensions
    const bool st2 = !grass(c, i) && c.rows[i] != p;
    g.E.emplace_back(sizeof(double) * (st2 ? 4 : 1) * p * p * c.rs);
    g.Q2.emplace_back(st2 ? sizeof(double) * c.rows[i] * p * c.rs : 0);
    g.P1.emplace_back(sizeof(double) * p * p * c.rs);
    g.P2.emplace_back(sizeof(double) * p * p * c.rs);
    g.Pc.emplace_back(sizeof(double) * p * p * c.rs);
  }
  const int m = std::max(1, cfg.lbfgs_m);
  for (int i = 0; i < m; ++i) {
    c.mem_s.emplace_back(tb);
    c.mem_y.emplace_back(tb);
  }
  c.dir.alloc(tb);
  c.dir2.alloc(tb);
  c.tmpv.alloc(tb);
  c.tmpv2.alloc(tb);
  std::vector<double> host(c.total, 0.0);
  for (int i = 0; i < c.nt; ++i)
    for (int64_t k = 0; k < std::min(c.rows[i], c.cols[i]); ++k)
      host[c.offs[i] + (k * c.cols[i] + k) * c.rs] = 1.0;
  MERA_CUDA(cudaMemcpyAsync(c.Wcur.p, host.data(), tb, cudaMemcpyHostToDevice, s));
  MERA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace
}  // namespace mera

// ================================================================ C ABI ====
using mera::Error;

namespace {
struct Guard {
  mera_t m;
  explicit Guard(mera_t mm) : m(mm) { mera::g_prof = mm ? &mm->prof : nullptr; }
  ~Guard() { mera::g_prof = nullptr; }
};

template <class F>
int wrap(mera_t m, F&& f) {
  Guard g(m);
  try {
    f();
    return MERA_OK;
  } catch (const Error& e) {
    if (m) m->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    if (m) m->err = "host allocation failed";
    return MERA_ERR_OOM;
  } catch (const std::exception& e) {
    if (m) m->err = e.what();
    return MERA_ERR_CUDA;
  }
}

void copy_in(mera_t m, const void* const* arr, double* flat) {
  for (int i = 0; i < m->nt; ++i) {
    if (!arr[i]) throw Error(MERA_ERR_ARG, "null tensor pointer");
    MERA_CUDA(cudaMemcpyAsync(flat + m->offs[i], arr[i], sizeof(double) * m->rows[i] * m->cols[i] * m->rs,
                              cudaMemcpyDefault, m->s));
  }
}
void copy_out(mera_t m, const double* flat, void* const* arr) {
  for (int i = 0; i < m->nt; ++i) {
    if (!arr[i]) throw Error(MERA_ERR_ARG, "null tensor pointer");
    MERA_CUDA(cudaMemcpyAsync(arr[i], flat + m->offs[i], sizeof(double) * m->rows[i] * m->cols[i] * m->rs,
                              cudaMemcpyDefault, m->s));
  }
  MERA_CUDA(cudaStreamSynchronize(m->s));
}
}  // namespace

extern "C" {

void mera_config_default(mera_config* c, int d_b, int chi, int n_trans) {
  std::memset(c, 0, sizeof(*c));
  c->d_b = d_b;
  c->chi = chi;
  c->n_trans = n_trans;
  c->dtype = MERA_F64;
  c->prec = MERA_PREC_FP64;
  c->w_stiefel = 0;
  c->precond = 1;
  c->krylov_dim = 20;
  c->krylov_maxiter = 2000;
  c->krylov_tol = 1e-14;
  c->recompute_env = 0;
  c->lbfgs_m = 8;
  c->b_chunk = 0;
  c->network = MERA_BINARY;
  c->z2 = 0;
}

int mera_create(const mera_config* cfg, const void* h3, void* stream, mera_t* out) {
  if (!cfg || !h3 || !out) return MERA_ERR_ARG;
  mera_t m = new (std::nothrow) mera_ctx();
  if (!m) return MERA_ERR_OOM;
  int rc = wrap(m, [&] { mera::create(*m, *cfg, h3, static_cast<cudaStream_t>(stream)); });
  if (rc != MERA_OK) {
    delete m;
    *out = nullptr;
    return rc;
  }
  *out = m;
  return MERA_OK;
}

int mera_destroy(mera_t m) {
  if (!m) return MERA_ERR_ARG;
  cudaStreamSynchronize(m->s);
  delete m;
  return MERA_OK;
}

int mera_num_tensors(mera_t m) { return m ? m->nt : MERA_ERR_ARG; }

int mera_tensor_shape(mera_t m, int i, int64_t* rows, int64_t* cols) {
  if (!m || i < 0 || i >= m->nt || !rows || !cols) return MERA_ERR_ARG;
  *rows = m->rows[i];
  *cols = m->cols[i];
  return MERA_OK;
}

int mera_set_tensors(mera_t m, const void* const* t) {
  if (!m || !t) return MERA_ERR_ARG;
  return wrap(m, [&] {
    copy_in(m, t, mera::P(m->Wtry));
    mera::check_isometric(*m, mera::P(m->Wtry), m->s);
    if (m->z2) mera::check_z2_point(*m, mera::P(m->Wtry), m->s);
    std::swap(m->Wcur, m->Wtry);
    m->ev[0].valid = m->ev[1].valid = false;
    mera::clear_history(*m);
    m->iters = 0;
  });
}

int mera_init_random(mera_t m, uint64_t seed) {
  if (!m) return MERA_ERR_ARG;
  return wrap(m, [&] {
    std::vector<double> host(m->total);
    for (int i = 0; i < m->nt; ++i) {
      std::vector<int> rq, cq;
      if (m->z2) {  // ternary: u_l (cf cf) x (cf cf), w_l (cf cf cf) x (cc)
        const int l = i / 2;
        const int64_t cf = m->dims[l], cc = l < m->L ? m->dims[l + 1] : m->dims[l];
        rq = mera::fused_charges(i % 2 == 0 ? std::vector<int64_t>{cf, cf} : std::vector<int64_t>{cf, cf, cf});
        cq = mera::fused_charges(i % 2 == 0 ? std::vector<int64_t>{cf, cf} : std::vector<int64_t>{cc});
      }
      mera::random_isometry(seed, (uint64_t)i, m->rows[i], m->cols[i], m->cplx, m->z2 ? rq.data() : nullptr,
                            m->z2 ? cq.data() : nullptr, host.data() + m->offs[i]);
    }
    MERA_CUDA(cudaMemcpyAsync(m->Wcur.p, host.data(), sizeof(double) * m->total, cudaMemcpyHostToDevice, m->s));
    MERA_CUDA(cudaStreamSynchronize(m->s));
    m->ev[0].valid = m->ev[1].valid = false;
    mera::clear_history(*m);
    m->iters = 0;
  });
}

int mera_get_tensors(mera_t m, void* const* t) {
  if (!m || !t) return MERA_ERR_ARG;
  return wrap(m, [&] { copy_out(m, mera::P(m->Wcur), t); });
}

int mera_energy(mera_t m, double* energy) {
  if (!m || !energy) return MERA_ERR_ARG;
  return wrap(m, [&] { *energy = mera::forward_energy(*m, mera::P(m->Wcur), m->s); });
}

int mera_energy_grad(mera_t m, double* energy, void* const* grad, void* const* deriv) {
  if (!m) return MERA_ERR_ARG;
  return wrap(m, [&] {
    mera::Eval& E = m->ev[m->cur];
    mera::energy_grad(*m, mera::P(m->Wcur), E, m->s);
    if (energy) *energy = E.e;
    if (grad) copy_out(m, mera::P(E.G), grad);
    if (deriv) copy_out(m, mera::P(E.D), deriv);
    MERA_CUDA(cudaStreamSynchronize(m->s));
  });
}

int mera_project(mera_t m, const void* const* D, void* const* G) {
  if (!m || !D || !G) return MERA_ERR_ARG;
  return wrap(m, [&] {
    copy_in(m, D, mera::P(m->tmpv));
    for (int i = 0; i < m->nt; ++i)
      mera::project_tensor(*m, i, mera::P(m->Wcur) + m->offs[i], mera::P(m->tmpv) + m->offs[i],
                           mera::P(m->tmpv2) + m->offs[i], m->s);
    copy_out(m, mera::P(m->tmpv2), G);
  });
}

int mera_inner(mera_t m, const void* const* X, const void* const* Y, double* out) {
  if (!m || !X || !Y || !out) return MERA_ERR_ARG;
  return wrap(m, [&] {
    copy_in(m, X, mera::P(m->tmpv));
    copy_in(m, Y, mera::P(m->tmpv2));
    *out = mera::inner(*m, mera::P(m->tmpv), mera::P(m->tmpv2), m->s);
  });
}

int mera_transport(mera_t m, const void* const* X, double alpha, void* const* Y) {
  if (!m || !X || !Y) return MERA_ERR_ARG;
  return wrap(m, [&] {
    copy_in(m, X, mera::P(m->dir2));
    copy_in(m, (const void* const*)Y, mera::P(m->tmpv));
    mera::make_geom(*m, mera::P(m->Wcur), mera::P(m->dir2), alpha, m->s);
    mera::apply_transport(*m, mera::P(m->Wcur), mera::P(m->dir2), mera::P(m->tmpv), m->s);
    copy_out(m, mera::P(m->tmpv), Y);
  });
}

int mera_retract(mera_t m, const void* const* X, double alpha, void* const* Xprime) {
  if (!m || !X) return MERA_ERR_ARG;
  return wrap(m, [&] {
    copy_in(m, X, mera::P(m->dir2));
    mera::make_geom(*m, mera::P(m->Wcur), mera::P(m->dir2), alpha, m->s);
    mera::apply_retract(*m, mera::P(m->Wcur), mera::P(m->dir2), mera::P(m->Wtry), m->s);
    if (Xprime) {
      mera::copy(mera::P(m->tmpv), mera::P(m->dir2), m->total, m->s);
      mera::apply_transport(*m, mera::P(m->Wcur), mera::P(m->dir2), mera::P(m->tmpv), m->s);
      copy_out(m, mera::P(m->tmpv), Xprime);
    }
    MERA_CUDA(cudaStreamSynchronize(m->s));
    std::swap(m->Wcur, m->Wtry);
    m->ev[0].valid = m->ev[1].valid = false;
    mera::clear_history(*m);
  });
}

int mera_precondition(mera_t m, const void* const* X, void* const* Xt) {
  if (!m || !X || !Xt) return MERA_ERR_ARG;
  return wrap(m, [&] {
    mera::Eval& E = m->ev[m->cur];
    if (!E.valid) throw Error(MERA_ERR_ARG, "mera_precondition needs a prior mera_energy_grad");
    copy_in(m, X, mera::P(m->tmpv));
    mera::precondition(*m, E, mera::P(m->Wcur), mera::P(m->tmpv), mera::P(m->tmpv2), m->s);
    copy_out(m, mera::P(m->tmpv2), Xt);
  });
}

int mera_lbfgs_step(mera_t m, mera_iter_info* info) {
  if (!m || !info) return MERA_ERR_ARG;
  return wrap(m, [&] { mera::lbfgs_step(*m, info, m->s); });
}

int mera_cg_step(mera_t m, mera_iter_info* info) {
  if (!m || !info) return MERA_ERR_ARG;
  return wrap(m, [&] { mera::cg_step(*m, info, m->s); });
}

int mera_ev_sweep(mera_t m, double gamma, mera_iter_info* info) {
  if (!m || !info || !std::isfinite(gamma)) return MERA_ERR_ARG;
  return wrap(m, [&] {
    std::memset(info, 0, sizeof(*info));
    mera::ev_sweep(*m, gamma, info, m->s);
  });
}

int mera_solve(mera_t m, const mera_solve_opts* o, mera_solve_result* r) {
  if (!m || !o || !r) return MERA_ERR_ARG;
  return wrap(m, [&] {
    std::memset(r, 0, sizeof(*r));
    mera::ensure_current(*m, m->s);
    mera_iter_info info{};
    double gn = std::sqrt(mera::inner(*m, mera::P(m->ev[m->cur].G), mera::P(m->ev[m->cur].G), m->s));
    r->n_evals = 1;
    for (int it = 0; it < o->maxiter && !(gn < o->gtol); ++it) {
      if (o->method == 1) mera::cg_step(*m, &info, m->s);
      else mera::lbfgs_step(*m, &info, m->s);
      gn = info.gnorm;
      r->iters++;
      r->n_evals += info.n_evals;
    }
    r->energy = m->ev[m->cur].e;
    r->gnorm = gn;
    r->converged = gn < o->gtol;
  });
}

namespace {
// mera_footprint_bytes for a uniform MPS (mirror of create_mps and the shared buffers)
size_t footprint_mps(const mera_config* cfg) {
  if (cfg->d_b < 2 || cfg->chi < 1 || cfg->n_trans != 0 || cfg->prec != MERA_PREC_FP64 || cfg->w_stiefel) return 0;
  const size_t rs = cfg->dtype == MERA_C128 ? 2 : 1, D = cfg->chi, d = cfg->d_b;
  const size_t n = D * D * rs;                  // reals of a D x D matrix
  const size_t total = D * d * D * rs;          // reals of the tensor
  const size_t q = D * rs;                      // order of the (embedded) eigenproblems
  size_t bytes = n + 3 * D * d * d * D * rs + total + 3 * n;             // rho, B, HB, T, scratch, h_l, h_r, H_l
  bytes += d * d * d * d * rs;                                           // h
  bytes += n * (size_t)(std::max(2, cfg->krylov_dim) + 1 + 3);           // Krylov basis, tmp, x, bvec
  bytes += 6 * D * d * D * rs * rs;                                      // geometry temporaries
  bytes += 2 * (n + q * q + q) + 2 * q * q + 4 * n;                      // evaluations' rho/eig, step geometry
  bytes += total * (size_t)(2 * std::max(1, cfg->lbfgs_m) + 2 + 4 + 4);  // memory, points, directions, G/D
  return 8 * bytes;
}

// mera_footprint_bytes for the ternary network
size_t footprint_ternary(const mera_config* cfg) {
  std::vector<int64_t> dims{cfg->d_b};
  for (int l = 0; l < cfg->n_trans; ++l) {
    const int64_t d = dims.back();
    dims.push_back(std::min<int64_t>(cfg->chi, d * d * d));
  }
  if (dims.back() != cfg->chi) return 0;
  const bool mixed = cfg->prec != MERA_PREC_FP64;
  const size_t rs = cfg->dtype == MERA_C128 ? 2 : 1;
  const size_t es = (mixed ? 4 : 8) * rs;
  mera::TablePool pool(true);
  size_t bytes = 0, ws = 0, total = 0, gmax = 1;
  for (size_t l = 0; l < dims.size(); ++l) {
    const int64_t cf = dims[l], cc = l + 1 < dims.size() ? dims[l + 1] : dims[l];
    total += (cf * cf * cf * cf + cf * cf * cf * cc) * rs;
    bytes += 2 * 8 * rs * (size_t)mera::ipow(cf, 4);  // h_l, rho_l
    gmax = std::max<size_t>({gmax, (size_t)(cf * cf * cf * cf), (size_t)(cc * cc * cc * cc),
                             (size_t)(cf * cf * cc * cc * cc), (size_t)(cf * cc * cc * cf),
                             (size_t)(cf * cc * cf * cf * cf), (size_t)(cf * cf * cf * cc),
                             (size_t)(cf * cf * cf * cc * cc * cc), (size_t)(cf * cf * cf * cf * cf * cc)});
    for (char sd : {'L', 'C', 'R'}) {
      mera::Net net(mera::ternary_netdef(sd), cf, cc, pool);
      for (int node = net.nleaf(); node < net.nnode(); ++node)
        bytes += es * (size_t)net.size(node) * (node == net.root() ? 1 : 2);
      for (const mera::GemmPlan* p : net.plans()) ws = std::max(ws, mera::tc_workspace_bytes(p->proto, cfg->prec));
    }
  }
  const size_t nS = (size_t)mera::ipow(cfg->chi, 4) * rs;
  bytes += ws + pool.bytes();
  bytes += 8 * nS * (size_t)(std::max(2, cfg->krylov_dim) + 1 + 3);  // basis, tmp, x, bvec
  bytes += 8 * gmax * 6 * rs * rs;
  bytes += 8 * (size_t)total * (size_t)(2 * std::max(1, cfg->lbfgs_m) + 2 + 4 + 4);
  return bytes;
}
}  // namespace

size_t mera_footprint_bytes(const mera_config* cfg) {
  if (!cfg) return 0;
  if (cfg->z2 != 0 && (cfg->z2 != 1 || cfg->network != MERA_TERNARY)) return 0;
  if (cfg->network == MERA_MPS) return footprint_mps(cfg);
  if (cfg->d_b < 2 || cfg->chi < 2 || cfg->n_trans < 1) return 0;
  if (cfg->network == MERA_TERNARY) {
    try {
      return footprint_ternary(cfg);
    } catch (...) {
      return 0;
    }
  }
  if (cfg->network != MERA_BINARY) return 0;
  try {
    // mirror of the allocations made by mera_create, with plans built dry
    std::vector<int64_t> dims{cfg->d_b};
    for (int l = 0; l < cfg->n_trans; ++l) dims.push_back(std::min<int64_t>(cfg->chi, dims.back() * dims.back()));
    if (dims.back() != cfg->chi) return 0;
    const bool mixed = cfg->prec != MERA_PREC_FP64;
    const size_t rs = cfg->dtype == MERA_C128 ? 2 : 1;
    const size_t es = (mixed ? 4 : 8) * rs;
    mera::TablePool pool(true);
    size_t bytes = 0, scratch = 0, ws = 0, total = 0, gmax = 1, keep[2] = {0, 0}, dep_max[3] = {0, 0, 0};
    for (size_t l = 0; l < dims.size(); ++l) {
      const int64_t cf = dims[l], cc = l + 1 < dims.size() ? dims[l + 1] : dims[l];
      int64_t chunk = mera::choose_chunk(cf, cc);
      if (cfg->b_chunk > 0) chunk = cfg->b_chunk < cc ? cfg->b_chunk : 0;
      total += (cf * cf * cf * cf + cf * cf * cc) * rs;
      bytes += 2 * 8 * rs * (size_t)mera::ipow(cf, 6);  // h_l, rho_l
      gmax = std::max<size_t>({gmax, (size_t)(cf * cf * cf * cf), (size_t)(cc * cc * cc * cc),
                               (size_t)(cf * cf * cc * cc * cc), (size_t)(cf * cc * cc * cf),
                               (size_t)(cf * cc * cf * cf * cf)});
      for (char sd : {'L', 'R'}) {
        mera::SideNet net(sd, cf, cc, pool, chunk);
        for (int node : {11, 13, 14, 16, 17, 18, 19}) {
          if (cfg->recompute_env && (node == 13 || node == 17 || node == 18)) {
            const int k = node == 13 ? 0 : node == 17 ? 1 : 2;
            dep_max[k] = std::max<size_t>(dep_max[k], net.alloc_size(node));
            continue;
          }
          bytes += es * net.alloc_size(node);
        }
        size_t need = 0;
        for (int node : {12, 15}) need += net.alloc_size(node);
        for (int node = 11; node < 20; ++node) need += net.alloc_size(node);
        scratch = std::max(scratch, es * need);
        for (const mera::GemmPlan* p : net.executed_plans())
          ws = std::max(ws, mera::tc_workspace_bytes(p->proto, cfg->prec));
        size_t kn[2];
        mera::keep_need(net, cfg->prec, kn);
        keep[0] = std::max(keep[0], kn[0]);
        keep[1] = std::max(keep[1], kn[1]);
      }
    }
    const size_t nS = (size_t)mera::ipow(cfg->chi, 6) * rs;
    bytes += es * (dep_max[0] + dep_max[1] + dep_max[2]);  // shared N3, N7, N8 (recomputation)
    bytes += scratch + ws + keep[0] + keep[1] + pool.bytes();
    bytes += 8 * nS * (size_t)(std::max(2, cfg->krylov_dim) + 1 + 3);  // basis, tmp, x, bvec
    bytes += 8 * gmax * 6 * rs * rs;
    bytes += 8 * (size_t)total * (size_t)(2 * std::max(1, cfg->lbfgs_m) + 2 + 4 + 4);
    return bytes;
  } catch (...) {
    return 0;
  }
}

int64_t mera_launch_count(mera_t m) { return m ? m->prof.launches : 0; }

int mera_get_stats(mera_t m, mera_stats* out, int reset) {
  if (!m || !out) return MERA_ERR_ARG;
  return wrap(m, [&] {
    MERA_CUDA(cudaStreamSynchronize(m->s));
    m->prof.collect();
    out->launches = m->prof.launches;
    out->gett_launches = m->prof.gett_launches;
    out->gett_flops = m->prof.gett_flops;
    out->gett_timed = m->prof.gett_timed;
    out->gett_ms = m->prof.gett_ms;
    out->energy_grad_calls = m->prof.energy_grad_calls;
    out->krylov_matvecs = m->matvecs;
    if (reset) {
      m->prof.shapes.clear();
      m->prof.launches = m->prof.gett_launches = m->prof.gett_timed = 0;
      m->prof.gett_flops = m->prof.gett_ms = 0.0;
      m->prof.energy_grad_calls = 0;
      m->matvecs = 0;
    }
  });
}

int mera_profile(mera_t m, int enable) {
  if (!m) return MERA_ERR_ARG;
  return wrap(m, [&] {
    MERA_CUDA(cudaStreamSynchronize(m->s));
    m->prof.collect();
    m->prof.timing = enable != 0;
  });
}

int mera_profile_dump(mera_t m, const char* path) {
  if (!m || !path) return MERA_ERR_ARG;
  return wrap(m, [&] {
    MERA_CUDA(cudaStreamSynchronize(m->s));
    m->prof.collect();
    FILE* f = std::fopen(path, "w");
    if (!f) throw Error(MERA_ERR_ARG, std::string("cannot write ") + path);
    std::fprintf(f, "M,N,K,path,calls,ms,tflops\n");
    for (const auto& kv : m->prof.shapes) {
      const auto& k = kv.first;
      const double fl = 2.0 * (double)k[0] * (double)k[1] * (double)k[2] * (double)kv.second.calls;
      std::fprintf(f, "%lld,%lld,%lld,%lld,%lld,%.4f,%.2f\n", (long long)k[0], (long long)k[1], (long long)k[2],
                   (long long)k[3], (long long)kv.second.calls, kv.second.ms,
                   kv.second.ms > 0 ? fl / (kv.second.ms * 1e9) : 0.0);
    }
    std::fclose(f);
  });
}

const char* mera_strerror(int code) {
  switch (code) {
    case MERA_OK: return "ok";
    case MERA_ERR_ARG: return "invalid argument";
    case MERA_ERR_OOM: return "out of device memory";
    case MERA_ERR_NONFINITE: return "non-finite energy or gradient";
    case MERA_ERR_NOCONV: return "iteration did not converge";
    case MERA_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case MERA_ERR_NOT_ISOMETRIC: return "tensor is not isometric";
    case MERA_ERR_CUDA: return "CUDA runtime error";
    case MERA_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

const char* mera_last_error(mera_t m) { return m ? m->err.c_str() : ""; }

int mera_gemm(int prec, int64_t M, int64_t N, int64_t K, const double* A, const double* B, double* C,
              void* stream) {
  if (M < 0 || N < 0 || K < 1 || !A || !B || !C) return MERA_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return wrap(nullptr, [&] {
    if (prec == MERA_PREC_FP64) {
      mera::gemm_f64('N', 'N', M, N, K, 1.0, A, K, B, N, 0.0, C, N, s);
      MERA_CUDA(cudaStreamSynchronize(s));
      return;
    }
    if (prec != MERA_PREC_3XTF32 && prec != MERA_PREC_SPLIT_BF16) throw Error(MERA_ERR_ARG, "bad precision");
    const int kind = prec == MERA_PREC_3XTF32 ? mera::tc::KIND_TF32 : mera::tc::KIND_BF16;
    const int elem = kind == mera::tc::KIND_TF32 ? 4 : 2;
    const int64_t Kp = mera::tc::padded_k(K, kind);
    const int64_t Mp = mera::tc::round_up(std::max<int64_t>(M, 1), 128), Np = mera::tc::round_up(std::max<int64_t>(N, 1), 128);
    mera::DevBuf ah(elem * Mp * Kp), al(elem * Mp * Kp), bh(elem * Np * Kp), bl(elem * Np * Kp), err(sizeof(int));
    const size_t skb = mera::tc::splitk_bytes(M, N, Kp, kind);
    mera::DevBuf part(skb);
    MERA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    mera::tc::pack_split(A, true, nullptr, K, nullptr, 1, M, K, Mp, Kp, kind, ah.p, al.p, false, s);
    mera::tc::pack_split(B, true, nullptr, 1, nullptr, N, N, K, Np, Kp, kind, bh.p, bl.p, true, s);
    mera::tc::TcEpilogue ep;
    ep.C = C;
    ep.c_f64 = 1;
    ep.cms = N;
    ep.cns = 1;
    ep.rows = N == 1;
    ep.err = err.as<int>();
    mera::tc::gemm_packed(kind, M, N, Kp, ah.p, al.p, Mp, bh.p, bl.p, Np, ep, s, part.as<float>(), skb);
    int e = 0;
    MERA_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MERA_CUDA(cudaStreamSynchronize(s));
    if (e) throw Error(MERA_ERR_DEVICE_TIMEOUT, "tensor-core GEMM: a bounded wait expired");
  });
}

}  // extern "C"
