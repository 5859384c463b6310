// libmera: scale-invariant MERA energy/gradient on one GPU (binary and
// ternary networks), and the problem's creation.  The geometry (geom.cu), the
// optimisers (optim.cu), the uniform MPS (mps.cu) and the C ABI (abi.cu) share
// the problem object of ctx.h.
//
//   energy_grad   (Sec. 4, App. B)
//     up-sweep    h_{l+1} = (A_L + A_R)(h_l)/2 through the transition layers
//     fixed point rho_S:  (1 - Dbar_S + |b><1|) rho = b, b = 1/chi^3, GMRES
//     series      x (1 - A') = <h_L|:  x - Abar_S(x) + Tr(x rho_S) 1 = h_L, GMRES
//     down-sweep  reverse pass of Tr(Abar_l(h_l) rho_{l+1}) per layer gives
//                 rho_l and the environments; the scale-invariant layer uses
//                 Tr(Abar_S(x) rho_S)
//     projection  Eqs. (stiefel_gradient), (grassmann_gradient)
//     rho_v       the density matrices of the preconditioner (Sec. 4)
//   creation      shapes, networks and buffers; input checks (isometry, Z2)
#include "ctx.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>

namespace mera {
thread_local Prof* g_prof = nullptr;

namespace {
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

}  // namespace

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

// Data-defined networks (tnet.h): the ternary network's three per layer (no
// intermediate above chi^6), or the binary network's two for Z2-symmetric
// problems (unsliced chains only); every internal node value and adjoint in
// its own buffer.
void build_layers_net(Ctx& c) {
  const bool mixed = c.cfg.prec != MERA_PREC_FP64;
  const size_t es = (mixed ? sizeof(float) : sizeof(double)) * c.rs;
  size_t ws_need = 0;
  for (int l = 0; l <= c.L && !c.tern; ++l) {
    const int64_t cf = c.dims[l], cc = l < c.L ? c.dims[l + 1] : c.dims[l];
    if (choose_chunk(cf, cc) != 0 || (c.cfg.b_chunk > 0 && c.cfg.b_chunk < cc))
      throw Error(MERA_ERR_UNSUPPORTED, "Z2 charge sectors of the binary network need an unsliced chain (chi <= 16)");
  }
  for (int l = 0; l <= c.L; ++l) {
    Layer& ly = c.layers[l];
    ly.cf = c.dims[l];
    ly.cc = l < c.L ? c.dims[l + 1] : c.dims[l];
    for (int sd = 0; sd < c.nsides; ++sd) {
      ly.tnet[sd] = std::make_unique<Net>(c.tern ? ternary_netdef("LCR"[sd]) : binary_netdef("LR"[sd]), ly.cf, ly.cc,
                                          c.pool, c.z2);
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
    c.ex.wait_ns = (uint64_t)(c.cfg.device_wait_s * 1e9);
  }
}

void bind_net(Layer& ly, int sd, const double* op, const double* u, const double* w) {
  NetBufs& b = ly.tbuf[sd];
  const Net& net = *ly.tnet[sd];
  for (int i = 0; i < net.nleaf(); ++i) {
    const int r = net.role(i);
    b.leaf[i] = r == ROLE_OP ? op : (r == ROLE_U || r == ROLE_UB) ? u : w;
  }
}

void build_layers(Ctx& c) {
  c.layers.resize(c.L + 1);
  if (c.gnet) {
    build_layers_net(c);
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
      if (c.cfg.prec == MERA_PREC_SPLIT_FP16) {
        ly.amax[sd].alloc(2 * SideNet::NNODE * sizeof(unsigned));
        MERA_CUDA(cudaMemsetAsync(ly.amax[sd].p, 0, ly.amax[sd].bytes, c.s));
        ly.buf[sd].amax = ly.amax[sd].as<unsigned>();
      }
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
    c.ex.wait_ns = (uint64_t)(c.cfg.device_wait_s * 1e9);
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
    c.have_rho = c.have_x = false;  // the Krylov vectors may hold an aborted product's garbage
    throw Error(MERA_ERR_DEVICE_TIMEOUT, "tensor-core contraction: a bounded device-side wait expired");
  }
}

// -------------------------------------------------------- superoperators ---
// out = ao * out + af * Abar(op) (both sides), using layer l's tensors from point W.
void ascend(Ctx& c, int l, const double* W, const double* op, double* out, double af, cudaStream_t s) {
  Layer& ly = c.layers[l];
  const double* u = W + c.offs[2 * l];
  const double* w = W + c.offs[2 * l + 1];
  if (c.gnet) {  // Abar = the average of the nsides maps
    for (int sd = 0; sd < c.nsides; ++sd) {
      bind_net(ly, sd, op, u, w);
      net_forward(*ly.tnet[sd], ly.tbuf[sd], out, af / c.nsides, 1.0, s);
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
  if (c.gnet) {
    for (int sd = 0; sd < c.nsides; ++sd) {
      bind_net(ly, sd, nullptr, u, w);
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
  if (c.gnet) {  // Dbar = the average of the nsides adjoint maps; needs only the prepared values
    for (int sd = 0; sd < c.nsides; ++sd)
      net_backward(*ly.tnet[sd], ly.tbuf[sd], r, true, out, af / c.nsides, false, nullptr, nullptr, 0.0, s);
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
  // mixed modes: a cycle whose residual estimate meets the target ends the
  // solve (see trust_estimate)
  const bool trust = trust_estimate(c.cfg.prec);
  while (true) {
    op(x, w);
    ++applications;
    axpby(1.0, b, -1.0, w, n, s);  // w = b - A x
    const double beta = std::sqrt(c.red.dot(w, w, n, s));
    // an expired tensor-core wait leaves garbage in w: stop at once
    check_device_flag(c, s);
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
    bool est_ok = false;
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
      est_ok = std::fabs(g[j + 1]) <= 0.5 * tol * bnorm;
      if (est_ok || hn == 0.0 || applications >= maxit) {
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
    if (trust && est_ok) {
      check_device_flag(c, s);
      return applications;
    }
  }
}

// --------------------------------------------------------- energy / grad ---
// The relative residual a Krylov solve can reach is limited by the rounding
// of the contractions that apply the superoperator: targets below this floor
// are raised to it.
// In the mixed modes the solves' target is the operator's own rounding
// level (krylov_floor), so a residual computed anew after a cycle measures
// that rounding rather than the solve: a cycle whose GMRES residual estimate
// meets half the target ends the solve without that extra application.  The
// FP64 path, whose target lies near the arithmetic's limit where the estimate
// can run ahead of the true residual, confirms every cycle's residual.
bool trust_estimate(int prec) { return prec != MERA_PREC_FP64; }

double krylov_floor(int prec) {
  // 22-bit modes: 2e-6, below the derivative error their tensor-core
  // accumulation leaves (4e-6 relative, measured at chi <= 12); a tighter
  // target changes neither the energy nor the derivatives (measured)
  const double f = prec == MERA_PREC_3XTF32 || prec == MERA_PREC_SPLIT_FP16 ? 2e-6
                   : prec == MERA_PREC_SPLIT_BF16                         ? 2e-5
                                                                          : 0.0;
  return f;
}

void project_tensor(Ctx& c, int i, const double* W, const double* D, double* G, cudaStream_t s) {
  const int64_t n = c.rows[i], p = c.cols[i];
  double* S = P(c.gtmp[0]);
  mm(c, 'C', 'N', p, p, n, 1.0, W, p, D, p, 0.0, S, p, s);     // S = W^dag D
  const bool stiefel = !grass(c, i);
  if (stiefel) herm(c, S, p, s);                                // (S + S^dag)/2
  if (G != D) copy(G, D, n * p * c.rs, s);
  mm(c, 'N', 'N', n, p, p, -1.0, W, p, S, p, 1.0, G, p, s);    // G = D - W S
}

void compute_rho_v(Ctx& c, Eval& E, const double* W, cudaStream_t s);
void gradient_pass(Ctx& c, const double* W, Eval& E, cudaStream_t s);

// Energy only: up-sweep, scale-invariant fixed point, e = Tr(h_L rho_S).
double forward_energy(Ctx& c, const double* W, cudaStream_t s);

bool grouped_eval(const Ctx& c) { return !c.gnet && !c.mps && !c.cplx; }

namespace {
// A single problem on the lockstep path: a group of one.
void eval_single(Ctx& c, const double* W, Eval& E, bool grad, cudaStream_t s) {
  Ctx* cs[1] = {&c};
  const double* Ws[1] = {W};
  Eval* Es[1] = {&E};
  std::exception_ptr err[1];
  eval_group(cs, Ws, Es, 1, grad, c.ex, s, err);
  if (err[0]) std::rethrow_exception(err[0]);
}
}  // namespace

// Full evaluation at point W into E.
void energy_grad(Ctx& c, const double* W, Eval& E, cudaStream_t s) {
  if (c.cohort_eval) {
    c.cohort_eval(c.cohort, c, W, E);
    return;
  }
  if (grouped_eval(c)) {
    eval_single(c, W, E, true, s);
    return;
  }
  const int L = c.L;
  c.prof.energy_grad_calls++;
  if (c.mps) {
    mps_energy_grad(c, W, E, s);
    return;
  }
  E.e = forward_energy(c, W, s);
  const int64_t cS = c.dims[L], n3 = opn(c, cS), n = n3 * n3;
  const double tol = std::max(c.cfg.krylov_tol, krylov_floor(c.cfg.prec));
  double* rhoS = P(c.rho[L]);
  double* hL = P(c.h[L]);
  double* xs = P(c.x);
  const int64_t nr = n * c.rs;  // reals per chi^6 operator
  // the warm start counts as valid again only once this solve has succeeded
  // (a solve that throws may leave x partly updated or non-finite)
  if (!c.have_x) copy(xs, hL, nr, s);
  c.have_x = false;
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
  if (grouped_eval(c)) {
    Eval e;  // receives the energy only
    eval_single(c, W, e, false, s);
    return e.e;
  }
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
  c.have_rho = false;  // set again once the solve below has produced a finite fixed point
  double* bvec = P(c.bvec);
  fill(0.0, bvec, nr, s);
  add_id(c, 1.0 / (double)n3, bvec, n3, s);
  // the residual of a Krylov solve cannot fall below the rounding level of
  // the contractions that apply the superoperator
  const double tol = std::max(c.cfg.krylov_tol, krylov_floor(c.cfg.prec));
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
  // Tr(h rho) = Re sum_ij h_ij conj(rho_ij): the real dot product of the arrays
  const double e = c.red.dot(P(c.h[L]), rhoS, nr, s);
  check_device_flag(c, s);
  if (!std::isfinite(e)) throw Error(MERA_ERR_NONFINITE, "non-finite energy");
  c.have_rho = true;
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
    for (int sd = 0; c.gnet && sd < c.nsides; ++sd) {
      // D_v = 2 dC/d conj(v) with C = Tr(Abar(h) rho), Abar the average of the nsides maps
      bind_net(ly, sd, op, u, w);
      if (l == L || c.cfg.recompute_env) net_forward(*ly.tnet[sd], ly.tbuf[sd], nullptr, 0.0, 0.0, s);
      net_backward(*ly.tnet[sd], ly.tbuf[sd], r, need_op, need_op ? P(c.rho[l]) : nullptr, 1.0 / c.nsides, true,
                   D + c.offs[2 * l], D + c.offs[2 * l + 1], 2.0 / c.nsides, s);
    }
    for (int sd = 0; !c.gnet && sd < 2; ++sd) {
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

// ------------------------------------------------------------ creation -----
void check_isometric(Ctx& c, const double* W, cudaStream_t s) {
  for (int i = 0; i < c.nt; ++i) {
    const int64_t n = c.rows[i], p = c.cols[i];
    double* S = P(c.gtmp[0]);
    mm(c, 'C', 'N', p, p, n, 1.0, W + c.offs[i], p, W + c.offs[i], p, 0.0, S, p, s);
    add_id(c, -1.0, S, p, s);
    const double r = std::sqrt(c.red.dot(S, S, p * p * c.rs, s));
    // a NaN or infinite entry of W makes W^dag W - 1 non-finite
    if (!std::isfinite(r)) throw Error(MERA_ERR_NONFINITE, "tensor " + std::to_string(i) + " has a non-finite entry");
    if (!(r < 1e-10)) throw Error(MERA_ERR_NOT_ISOMETRIC, "tensor " + std::to_string(i) + " has |W^T W - 1| = " + std::to_string(r));
  }
}

void create_mera(Ctx& c, int64_t* nS, int64_t* gmax);
void finish_create(Ctx& c, cudaStream_t s);

std::string config_range_error(const mera_config& cfg) {
  auto flag = [](int v) { return v == 0 || v == 1; };
  if (!flag(cfg.w_stiefel) || !flag(cfg.precond) || !flag(cfg.recompute_env) || !flag(cfg.z2))
    return "w_stiefel, precond, recompute_env and z2 must be 0 or 1";
  if (!(cfg.krylov_tol > 0.0 && cfg.krylov_tol < 1.0)) return "need 0 < krylov_tol < 1";
  if (cfg.krylov_maxiter < 1 || cfg.krylov_dim < 1 || cfg.lbfgs_m < 1) return "need krylov_maxiter, krylov_dim, lbfgs_m >= 1";
  if (cfg.b_chunk < 0) return "need b_chunk >= 0";
  if (!(cfg.device_wait_s > 0.0 && cfg.device_wait_s <= 60.0)) return "need 0 < device_wait_s <= 60";
  return "";
}

// The Hamiltonian term (n x n on the device) must be Hermitian: |h - h^dag|
// at most 1e-10 of its largest entry, else MERA_ERR_ARG (MERA_ERR_NONFINITE
// for a NaN or infinite entry).
void check_hermitian(Ctx& c, const double* dev, int64_t n, cudaStream_t s) {
  std::vector<double> h((size_t)(n * n * c.rs));
  MERA_CUDA(cudaMemcpyAsync(h.data(), dev, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  double big = 0.0, bad = 0.0;
  for (const double x : h)
    if (!std::isfinite(x)) throw Error(MERA_ERR_NONFINITE, "the Hamiltonian term is not finite");
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      const double* a = h.data() + (i * n + j) * c.rs;
      const double* b = h.data() + (j * n + i) * c.rs;
      const double dr = a[0] - b[0], di = c.cplx ? a[1] + b[1] : 0.0;  // h_ij - conj(h_ji)
      big = std::max(big, c.cplx ? std::hypot(a[0], a[1]) : std::fabs(a[0]));
      bad = std::max(bad, std::hypot(dr, di));
    }
  if (bad > 1e-10 * big)
    throw Error(MERA_ERR_ARG, "the Hamiltonian term is not Hermitian (|h - h^dag| = " + std::to_string(bad) + ")");
}

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

// Z2 symmetry of a (rows x cols) matrix on the device whose rows (columns)
// are index tuples of legs with dimensions rdims (cdims), row-major: every
// entry between a row and a column of different total charge (the legs'
// gradings summed, first half of each leg even) must be below 1e-12 of the
// largest entry (Sec. 6); MERA_ERR_ARG otherwise.
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

// Legs of the rows and columns of tensor i of a MERA point: u_l (cf cf) x
// (cf cf), w_l (cf cf) x (cc) binary or (cf cf cf) x (cc) ternary.
void tensor_legs(const Ctx& c, int i, std::vector<int64_t>& rows, std::vector<int64_t>& cols) {
  const int l = i / 2;
  const int64_t cf = c.dims[l], cc = l < c.L ? c.dims[l + 1] : c.dims[l];
  if (i % 2 == 0) {
    rows = cols = {cf, cf};
  } else {
    rows.assign(c.tern ? 3 : 2, cf);
    cols = {cc};
  }
}

// Z2 symmetry of every tensor of a MERA point.
void check_z2_point(Ctx& c, const double* W, cudaStream_t s) {
  for (int i = 0; i < c.nt; ++i) {
    std::vector<int64_t> rows, cols;
    tensor_legs(c, i, rows, cols);
    check_z2(c, W + c.offs[i], rows, cols, (i % 2 == 0 ? "u_" : "w_") + std::to_string(i / 2), s);
  }
}

void create(Ctx& c, const mera_config& cfg, const void* h3, cudaStream_t s) {
  c.cfg = cfg;
  c.s = s;
  if (cfg.dtype != MERA_F64 && cfg.dtype != MERA_C128) throw Error(MERA_ERR_ARG, "unknown dtype");
  c.cplx = cfg.dtype == MERA_C128;
  c.rs = c.cplx ? 2 : 1;
  if (cfg.prec < MERA_PREC_FP64 || cfg.prec > MERA_PREC_SPLIT_FP16)
    throw Error(MERA_ERR_ARG, "unknown precision mode");
  if (cfg.network != MERA_BINARY && cfg.network != MERA_TERNARY && cfg.network != MERA_MPS)
    throw Error(MERA_ERR_ARG, "unknown network");
  const std::string bad = config_range_error(cfg);
  if (!bad.empty()) throw Error(MERA_ERR_ARG, bad);
  c.tern = cfg.network == MERA_TERNARY;
  c.mps = cfg.network == MERA_MPS;
  if (cfg.z2 != 0 && cfg.z2 != 1) throw Error(MERA_ERR_ARG, "z2 must be 0 or 1");
  c.z2 = cfg.z2 == 1;
  if (c.z2 && c.mps) throw Error(MERA_ERR_UNSUPPORTED, "Z2 charge sectors are built for the MERA networks");
  c.gnet = c.tern || c.z2;
  c.nsides = c.tern ? 3 : 2;
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
  check_hermitian(c, P(c.h0), ipow(cfg.d_b, c.ns), s);
  if (c.z2) {
    const std::vector<int64_t> sites(c.ns, cfg.d_b);
    check_z2(c, P(c.h0), sites, sites, "the Hamiltonian term", s);
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

}  // namespace mera
