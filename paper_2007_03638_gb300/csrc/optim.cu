// The optimisers (Sec. 3): Hager-Zhang line search, L-BFGS two-loop,
// nonlinear conjugate gradient, and the Evenbly-Vidal sweeps they are
// compared against (App. ev_steplimit).
#include "ctx.h"

#include <cmath>

namespace mera {

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
  spectral_values(f, (int)q, 5, 0.0, 1e-300, fr, s);
  v_diag_vt(V, fr, (int)q, c.cplx ? F : R, s);
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

// Riemannian gradient descent (Sec. 3): the direction -P(G), the
// Hager-Zhang step started at the previous accepted step.
void gd_step(Ctx& c, mera_iter_info* info, cudaStream_t s) {
  ensure_current(c, s);
  const int64_t mv0 = c.matvecs;
  Eval& E = c.ev[c.cur];
  const double* W = P(c.Wcur);
  double* G = P(E.G);
  double* d = P(c.dir);
  // the L-BFGS pairs and the CG direction are not transported by this step
  c.mem_n = 0;
  c.mem_rho.clear();
  precondition(c, E, W, G, d, s);
  scal(-1.0, d, c.total, s);
  const double df0 = inner(c, G, d, s);
  const double f0 = E.e;
  LsResult ls = hager_zhang(c, f0, df0, c.alpha_prev, s);
  info->n_evals = ls.nev;
  info->ls_ok = ls.ok;
  if (!ls.found || (!ls.ok && ls.f >= f0)) {
    info->alpha = 0.0;
    info->energy = f0;
    info->gnorm = std::sqrt(inner(c, G, G, s));
    info->iter = ++c.iters;
    info->krylov_matvecs = (int)(c.matvecs - mv0);
    return;
  }
  c.alpha_prev = ls.alpha;
  accept(c, s);
  Eval& En = c.ev[c.cur];
  info->alpha = ls.alpha;
  info->energy = En.e;
  info->gnorm = std::sqrt(inner(c, P(En.G), P(En.G), s));
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
  // Hager-Zhang's lower bound -1 / (|d_k| min(eta, |g_k|)): d_k the direction
  // just searched (transported; the transport is isometric), g_k the gradient
  // at the point it started from, eta = 0.01
  const double dn = std::sqrt(inner(c, d2, d2, s));
  const double gn_old = std::sqrt(inner(c, G, G, s));
  const double gn = std::sqrt(inner(c, P(En.G), P(En.G), s));
  beta = std::max(beta, -1.0 / (dn * std::min(0.01, gn_old)));
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

}  // namespace mera
