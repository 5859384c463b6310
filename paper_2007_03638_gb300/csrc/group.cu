// Energy and gradient of several problems of the same binary network at
// once (Sec. 4 with App. B), in lockstep: every pairwise contraction of the
// networks is one batched tensor-core launch over the members
// (contract_batch), the scale-invariant Krylov solves advance all members one
// operator application at a time, and the members' reductions of a round
// share one synchronisation.  Each member's arithmetic is that of the member
// evaluated alone (a group of one is the single-problem evaluation), so its
// results do not depend on the group it runs in.
#include "ctx.h"

#include <algorithm>
#include <cmath>
#include <exception>

namespace mera {
namespace {

struct Grp {
  Ctx* const* c;
  const double* const* W;
  Eval* const* E;
  int nb = 0;
  const Exec* ex = nullptr;  // workspace and wait flag of the batched products
  cudaStream_t s = nullptr;
  std::vector<int> alive;    // members still being evaluated
  std::vector<std::exception_ptr> err;
};

void fail_member(Grp& g, int k, std::exception_ptr e) {
  g.err[k] = e;
  g.c[k]->have_rho = g.c[k]->have_x = false;
  g.alive.erase(std::remove(g.alive.begin(), g.alive.end(), k), g.alive.end());
}

// f(k) for every member still alive; an exception fails that member only
template <class F>
void each(Grp& g, F f) {
  const std::vector<int> a = g.alive;
  for (int k : a) {
    try {
      f(k);
    } catch (...) {
      fail_member(g, k, std::current_exception());
    }
  }
}

// a step shared by all members (a batched launch): an exception fails them all
template <class F>
void together(Grp& g, F f) {
  try {
    f();
  } catch (...) {
    const std::exception_ptr e = std::current_exception();
    const std::vector<int> a = g.alive;
    for (int k : a) fail_member(g, k, e);
  }
}

const double* u_of(const Grp& g, int k, int l) { return g.W[k] + g.c[k]->offs[2 * l]; }
const double* w_of(const Grp& g, int k, int l) { return g.W[k] + g.c[k]->offs[2 * l + 1]; }

// An expired tensor-core wait in a batched product concerns every member.
void check_group_flag(Grp& g) {
  if (!g.ex->err || g.alive.empty()) return;
  int e = 0;
  together(g, [&] {
    MERA_CUDA(cudaMemcpyAsync(&e, g.ex->err, sizeof(int), cudaMemcpyDeviceToHost, g.s));
    MERA_CUDA(cudaStreamSynchronize(g.s));
    if (e) {
      MERA_CUDA(cudaMemsetAsync(g.ex->err, 0, sizeof(int), g.s));
      throw Error(MERA_ERR_DEVICE_TIMEOUT, "tensor-core contraction: a bounded device-side wait expired");
    }
  });
}

void sync(Grp& g) {
  together(g, [&] { MERA_CUDA(cudaStreamSynchronize(g.s)); });
}

// ---- batched superoperators over a list of members (indices into g) ----
void prepare_all(Grp& g, int l) {
  together(g, [&] {
    for (int sd = 0; sd < 2; ++sd) {
      SideBufs* bs[tc::TcEpilogue::MAXB];
      int n = 0;
      for (int k : g.alive) {
        Layer& ly = g.c[k]->layers[l];
        bind_leaves(ly, sd, nullptr, u_of(g, k, l), w_of(g, k, l));
        bs[n++] = &ly.buf[sd];
      }
      if (n) side_prepare_n(*g.c[g.alive[0]]->layers[l].net[sd], bs, n, *g.ex, g.s);
    }
  });
}

// out[k] += af * Abar(op[k]) for the members in `ms`
void ascend_members(Grp& g, const std::vector<int>& ms, int l, const double* const* op, double* const* out,
                    double af) {
  if (ms.empty()) return;
  for (int sd = 0; sd < 2; ++sd) {
    SideBufs* bs[tc::TcEpilogue::MAXB];
    double* o[tc::TcEpilogue::MAXB];
    int n = 0;
    for (int k : ms) {
      Layer& ly = g.c[k]->layers[l];
      bind_leaves(ly, sd, op[k], u_of(g, k, l), w_of(g, k, l));
      bs[n] = &ly.buf[sd];
      o[n++] = out[k];
    }
    side_forward_n(*g.c[ms[0]]->layers[l].net[sd], bs, n, *g.ex, o, 0.5 * af, 1.0, g.s);
  }
}

// out[k] += af * Dbar(r[k]) (operator-path reverse pass) for the members in `ms`
void descend_members(Grp& g, const std::vector<int>& ms, int l, const double* const* r, double* const* out,
                     double af) {
  if (ms.empty()) return;
  for (int sd = 0; sd < 2; ++sd) {
    SideBufs* bs[tc::TcEpilogue::MAXB];
    double* o[tc::TcEpilogue::MAXB];
    int n = 0;
    for (int k : ms) {
      Layer& ly = g.c[k]->layers[l];
      ly.buf[sd].adj[SideNet::ROOT] = const_cast<double*>(r[k]);
      bs[n] = &ly.buf[sd];
      o[n++] = out[k];
    }
    side_backward_n(*g.c[ms[0]]->layers[l].net[sd], bs, n, *g.ex, true, o, 0.5 * af, false, nullptr, nullptr, 0.0,
                    g.s);
  }
}

// ---- restarted GMRES, all members in lockstep ----
// Per member the steps, the classical Gram-Schmidt with one
// re-orthogonalisation, the Givens rotations and the stopping rules are
// those of gmres() in mera.cu; only the operator applications are batched,
// and the reductions the members have pending share one synchronisation.
struct GmresMember {
  const double* b = nullptr;
  double* x = nullptr;
  int64_t n = 0;
  double tol = 0.0, bnorm = 0.0, best = INFINITY;
  int m = 0, maxit = 0, apps = 0, j = 0;
  // APPLY: waiting for A x (restart) or A V_j; RES: residual norm pending;
  // P1, P2: first / second projection pending; NORM: |V_{j+1}| pending
  enum { DONE, APPLY, RES, P1, P2, NORM } state = DONE;
  bool restart = true;  // the next application is A x
  std::vector<double> H, cs, sn, gv, h1, h2, y;
};

// End of a cycle: back substitution, x += V y, next application A x.
void finish_cycle(GmresMember& q, Ctx& c, cudaStream_t s) {
  const int j = q.j, m = q.m;
  for (int i = j - 1; i >= 0; --i) {
    double t = q.gv[i];
    for (int k = i + 1; k < j; ++k) t -= q.H[i * m + k] * q.y[k];
    q.y[i] = q.H[i * m + i] != 0 ? t / q.H[i * m + i] : 0.0;
  }
  MERA_CUDA(cudaMemcpyAsync(c.kcoef.p, q.y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
  combine(P(c.kbasis), q.n, j, P(c.kcoef), q.x, q.n, 1.0, s);
  q.restart = true;
  q.state = GmresMember::APPLY;
}

// op(ms, in, out): out[k] = A_k in[k] for the members k in ms (batched)
template <class Op>
void gmres_group(Grp& g, std::vector<GmresMember>& st, Op op) {
  each(g, [&](int k) {
    GmresMember& q = st[k];
    Ctx& c = *g.c[k];
    q.m = std::max(2, c.cfg.krylov_dim);
    q.maxit = std::max(q.m, c.cfg.krylov_maxiter);
    q.H.assign((q.m + 1) * q.m, 0.0);
    q.cs.assign(q.m, 0.0);
    q.sn.assign(q.m, 0.0);
    q.gv.assign(q.m + 1, 0.0);
    q.h1.assign(q.m + 1, 0.0);
    q.h2.assign(q.m + 1, 0.0);
    q.y.assign(q.m, 0.0);
    c.red.dots_async(q.b, 0, 1, q.b, q.n, g.s);
  });
  sync(g);
  each(g, [&](int k) {
    GmresMember& q = st[k];
    q.bnorm = std::sqrt(g.c[k]->red.pinned_results()[0]);
    if (q.bnorm == 0.0) {
      fill(0.0, q.x, q.n, g.s);
      q.state = GmresMember::DONE;
      return;
    }
    q.restart = true;
    q.state = GmresMember::APPLY;
  });
  auto in_state = [&](int s) {
    std::vector<int> a;
    for (int k : g.alive)
      if (st[k].state == s) a.push_back(k);
    return a;
  };
  auto pending = [&] {
    for (int k : g.alive)
      if (st[k].state != GmresMember::DONE && st[k].state != GmresMember::APPLY) return true;
    return false;
  };
  for (std::vector<int> a = in_state(GmresMember::APPLY); !a.empty(); a = in_state(GmresMember::APPLY)) {
    // one operator application for every member that waits for one
    const double* in[tc::TcEpilogue::MAXB] = {};
    double* out[tc::TcEpilogue::MAXB] = {};
    for (int k : a) {
      GmresMember& q = st[k];
      Ctx& c = *g.c[k];
      double* V = P(c.kbasis);
      in[k] = q.restart ? q.x : V + (int64_t)q.j * q.n;
      out[k] = q.restart ? P(c.ktmp) : V + (int64_t)(q.j + 1) * q.n;
    }
    together(g, [&] { op(a, in, out); });
    each(g, [&](int k) {
      GmresMember& q = st[k];
      if (q.state != GmresMember::APPLY) return;
      Ctx& c = *g.c[k];
      ++q.apps;
      if (q.restart) {
        double* w = P(c.ktmp);
        axpby(1.0, q.b, -1.0, w, q.n, g.s);  // w = b - A x
        c.red.dots_async(w, 0, 1, w, q.n, g.s);
        q.state = GmresMember::RES;
      } else {
        double* V = P(c.kbasis);
        c.red.dots_async(V, q.n, q.j + 1, V + (int64_t)(q.j + 1) * q.n, q.n, g.s);
        q.state = GmresMember::P1;
      }
    });
    // the members' pending reductions, one synchronisation per round
    while (pending()) {
      sync(g);
      bool residual_round = false;
      for (int k : g.alive) residual_round = residual_round || st[k].state == GmresMember::RES;
      if (residual_round) check_group_flag(g);  // an aborted product leaves garbage: stop at once
      each(g, [&](int k) {
        GmresMember& q = st[k];
        if (q.state == GmresMember::DONE || q.state == GmresMember::APPLY) return;
        Ctx& c = *g.c[k];
        double* V = P(c.kbasis);
        double* vj1 = V + (int64_t)(q.j + 1) * q.n;
        const double* r = c.red.pinned_results();
        const int m = q.m;
        switch (q.state) {
          case GmresMember::RES: {
            const double beta = std::sqrt(r[0]);
            if (beta <= q.tol * q.bnorm) {
              q.state = GmresMember::DONE;
              return;
            }
            if (q.apps >= q.maxit || !(beta < 1e300))
              throw Error(MERA_ERR_NOCONV, "GMRES: relative residual " + std::to_string(beta / q.bnorm));
            if (beta > 0.9 * q.best && q.apps > 2 * m && beta <= 100.0 * q.tol * q.bnorm) {
              q.state = GmresMember::DONE;  // no progress over a restart cycle: at the rounding floor
              return;
            }
            q.best = std::min(q.best, beta);
            axpby(1.0 / beta, P(c.ktmp), 0.0, V, q.n, g.s);
            std::fill(q.gv.begin(), q.gv.end(), 0.0);
            q.gv[0] = beta;
            q.j = 0;
            q.restart = false;
            q.state = GmresMember::APPLY;
            return;
          }
          case GmresMember::P1: {
            for (int i = 0; i <= q.j; ++i) q.h1[i] = -r[i];
            MERA_CUDA(cudaMemcpyAsync(c.kcoef.p, q.h1.data(), sizeof(double) * (q.j + 1), cudaMemcpyHostToDevice,
                                      g.s));
            combine(V, q.n, q.j + 1, P(c.kcoef), vj1, q.n, 1.0, g.s);
            c.red.dots_async(V, q.n, q.j + 1, vj1, q.n, g.s);
            q.state = GmresMember::P2;
            return;
          }
          case GmresMember::P2: {
            for (int i = 0; i <= q.j; ++i) q.h2[i] = -r[i];
            MERA_CUDA(cudaMemcpyAsync(c.kcoef.p, q.h2.data(), sizeof(double) * (q.j + 1), cudaMemcpyHostToDevice,
                                      g.s));
            combine(V, q.n, q.j + 1, P(c.kcoef), vj1, q.n, 1.0, g.s);
            for (int i = 0; i <= q.j; ++i) q.H[i * m + q.j] = -(q.h1[i] + q.h2[i]);
            c.red.dots_async(vj1, 0, 1, vj1, q.n, g.s);
            q.state = GmresMember::NORM;
            return;
          }
          case GmresMember::NORM: {
            const int j = q.j;
            const double hn = std::sqrt(r[0]);
            q.H[(j + 1) * m + j] = hn;
            if (hn > 0) scal(1.0 / hn, vj1, q.n, g.s);
            for (int i = 0; i < j; ++i) {
              const double t = q.cs[i] * q.H[i * m + j] + q.sn[i] * q.H[(i + 1) * m + j];
              q.H[(i + 1) * m + j] = -q.sn[i] * q.H[i * m + j] + q.cs[i] * q.H[(i + 1) * m + j];
              q.H[i * m + j] = t;
            }
            const double aa = q.H[j * m + j], bb = q.H[(j + 1) * m + j];
            const double rr = std::hypot(aa, bb);
            q.cs[j] = rr > 0 ? aa / rr : 1.0;
            q.sn[j] = rr > 0 ? bb / rr : 0.0;
            q.H[j * m + j] = rr;
            q.H[(j + 1) * m + j] = 0.0;
            q.gv[j + 1] = -q.sn[j] * q.gv[j];
            q.gv[j] = q.cs[j] * q.gv[j];
            ++q.j;
            const bool est_ok = std::fabs(q.gv[j + 1]) <= 0.5 * q.tol * q.bnorm;
            if (est_ok || hn == 0.0 || q.apps >= q.maxit || q.j == m) {
              finish_cycle(q, c, g.s);
              // the mixed modes end on the estimate (trust_estimate); the
              // group's device flag is checked when the solve returns
              if (est_ok && trust_estimate(c.cfg.prec)) q.state = GmresMember::DONE;
            } else {
              q.state = GmresMember::APPLY;
            }
            return;
          }
          default:
            return;
        }
      });
    }
  }
}

// ---- the evaluation ----
// Scale-invariant fixed point (the members whose warm start is not valid
// start from 1/chi^3): rho_S with Dbar_S rho_S = rho_S, Tr rho_S = 1, solved as
// (1 - Dbar_S + |b)(1|) rho = b; then e = Tr(h_S rho_S).
void fixed_point(Grp& g) {
  std::vector<GmresMember> st(g.nb);
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    const int L = c.L;
    const int64_t n3 = opn(c, c.dims[L]), nr = n3 * n3 * c.rs;
    double* rhoS = P(c.rho[L]);
    if (!c.have_rho) {
      fill(0.0, rhoS, nr, g.s);
      add_id(c, 1.0 / (double)n3, rhoS, n3, g.s);
    }
    c.have_rho = false;  // set again once the solve below has produced a finite fixed point
    fill(0.0, P(c.bvec), nr, g.s);
    add_id(c, 1.0 / (double)n3, P(c.bvec), n3, g.s);
    st[k].b = P(c.bvec);
    st[k].x = rhoS;
    st[k].n = nr;
    st[k].tol = std::max(c.cfg.krylov_tol, krylov_floor(c.cfg.prec));
  });
  gmres_group(g, st, [&](const std::vector<int>& ms, const double* const* in, double* const* out) {
    const int L = g.c[ms[0]]->L;
    for (int k : ms) {
      Ctx& c = *g.c[k];
      const int64_t n3 = opn(c, c.dims[L]);
      copy(out[k], in[k], n3 * n3 * c.rs, g.s);
    }
    descend_members(g, ms, L, in, out, -1.0);
    // + Tr(v) b, b = 1/chi^3
    for (int k : ms) g.c[k]->red.trace_async(in[k], opn(*g.c[k], g.c[k]->dims[L]), g.s);
    MERA_CUDA(cudaStreamSynchronize(g.s));
    for (int k : ms) {
      Ctx& c = *g.c[k];
      const int64_t n3 = opn(c, c.dims[L]);
      axpy(c.red.pinned_results()[0], P(c.bvec), out[k], n3 * n3, g.s);
      ++c.matvecs;
    }
  });
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    c.red.trace_async(P(c.rho[c.L]), opn(c, c.dims[c.L]), g.s);
  });
  sync(g);
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    const int L = c.L;
    const int64_t n3 = opn(c, c.dims[L]), nr = n3 * n3 * c.rs;
    const double tr = c.red.pinned_results()[0];
    if (!(std::fabs(tr) > 0)) throw Error(MERA_ERR_NONFINITE, "fixed point has zero trace");
    double* rhoS = P(c.rho[L]);
    scal(1.0 / tr, rhoS, nr, g.s);
    herm(c, rhoS, n3, g.s);
    // Tr(h rho) = sum_ij h_ij rho_ij: the dot product of the arrays
    c.red.dots_async(P(c.h[L]), 0, 1, rhoS, nr, g.s);
  });
  sync(g);
  check_group_flag(g);
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    const double e = c.red.pinned_results()[0];
    if (!std::isfinite(e)) throw Error(MERA_ERR_NONFINITE, "non-finite energy");
    g.E[k]->e = e;
    c.have_rho = true;
  });
}

// Up-sweep (h_{l+1} = Abar(h_l)) and the fixed point.
void forward(Grp& g) {
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    copy(P(c.h[0]), P(c.h0), opn(c, c.dims[0]) * opn(c, c.dims[0]) * c.rs, g.s);
    if (c.hshift != 0.0) add_id(c, -c.hshift, P(c.h[0]), opn(c, c.dims[0]), g.s);
  });
  if (g.alive.empty()) return;
  const int L = g.c[g.alive[0]]->L;
  for (int l = 0; l <= L; ++l) prepare_all(g, l);
  for (int l = 0; l < L; ++l) {
    const double* op[tc::TcEpilogue::MAXB] = {};
    double* out[tc::TcEpilogue::MAXB] = {};
    each(g, [&](int k) {
      Ctx& c = *g.c[k];
      const int64_t n3 = opn(c, c.dims[l + 1]);
      fill(0.0, P(c.h[l + 1]), n3 * n3 * c.rs, g.s);
      op[k] = P(c.h[l]);
      out[k] = P(c.h[l + 1]);
    });
    together(g, [&] { ascend_members(g, g.alive, l, op, out, 1.0); });
    each(g, [&](int k) { herm(*g.c[k], P(g.c[k]->h[l + 1]), opn(*g.c[k], g.c[k]->dims[l + 1]), g.s); });
  }
  fixed_point(g);
}

// Environment series x = sum_i <h_S| A'^i (App. B): (1 - Abar_S + |1)(rho|) x = h_S.
void series(Grp& g) {
  std::vector<GmresMember> st(g.nb);
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    const int L = c.L;
    const int64_t n3 = opn(c, c.dims[L]), nr = n3 * n3 * c.rs;
    // the warm start counts as valid again only once this solve has succeeded
    if (!c.have_x) copy(P(c.x), P(c.h[L]), nr, g.s);
    c.have_x = false;
    st[k].b = P(c.h[L]);
    st[k].x = P(c.x);
    st[k].n = nr;
    st[k].tol = std::max(c.cfg.krylov_tol, krylov_floor(c.cfg.prec));
  });
  gmres_group(g, st, [&](const std::vector<int>& ms, const double* const* in, double* const* out) {
    const int L = g.c[ms[0]]->L;
    for (int k : ms) {
      Ctx& c = *g.c[k];
      const int64_t n3 = opn(c, c.dims[L]);
      copy(out[k], in[k], n3 * n3 * c.rs, g.s);
    }
    ascend_members(g, ms, L, in, out, -1.0);
    // + Tr(v rho) 1
    for (int k : ms) {
      Ctx& c = *g.c[k];
      const int64_t n3 = opn(c, c.dims[L]);
      c.red.dots_async(in[k], 0, 1, P(c.rho[L]), n3 * n3, g.s);
    }
    MERA_CUDA(cudaStreamSynchronize(g.s));
    for (int k : ms) {
      Ctx& c = *g.c[k];
      add_identity(c.red.pinned_results()[0], out[k], opn(c, c.dims[L]), g.s);
      ++c.matvecs;
    }
  });
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    herm(c, P(c.x), opn(c, c.dims[c.L]), g.s);
    c.have_x = true;
  });
}

// Reverse passes of every layer (environments, descending maps), projection
// and the preconditioner's density matrices.
void reverse(Grp& g) {
  each(g, [&](int k) { fill(0.0, P(g.E[k]->D), g.c[k]->total, g.s); });
  if (g.alive.empty()) return;
  const int L = g.c[g.alive[0]]->L;
  for (int l = L; l >= 0; --l) {
    const bool need_op = l < L;
    each(g, [&](int k) {
      Ctx& c = *g.c[k];
      const int64_t cf = c.layers[l].cf;
      if (need_op) fill(0.0, P(c.rho[l]), opn(c, cf) * opn(c, cf) * c.rs, g.s);
    });
    together(g, [&] {
      for (int sd = 0; sd < 2; ++sd) {
        SideBufs* bs[tc::TcEpilogue::MAXB];
        double *oo[tc::TcEpilogue::MAXB], *du[tc::TcEpilogue::MAXB], *dw[tc::TcEpilogue::MAXB];
        int n = 0;
        bool fwd = false;
        for (int k : g.alive) {
          Ctx& c = *g.c[k];
          Layer& ly = c.layers[l];
          const double* op = l < L ? P(c.h[l]) : P(c.x);
          bind_leaves(ly, sd, op, u_of(g, k, l), w_of(g, k, l));
          fwd = l == L || c.cfg.recompute_env;
          bs[n] = &ly.buf[sd];
          oo[n] = need_op ? P(c.rho[l]) : nullptr;
          du[n] = P(g.E[k]->D) + c.offs[2 * l];
          dw[n] = P(g.E[k]->D) + c.offs[2 * l + 1];
          ++n;
        }
        const SideNet& net = *g.c[g.alive[0]]->layers[l].net[sd];
        // the reverse pass needs N3, N7, N8 for this layer's operator: the
        // up-sweep left them in place for the transition layers (unless
        // recomputation was asked for); the scale-invariant layer's operator is x
        if (fwd) side_forward_n(net, bs, n, *g.ex, nullptr, 0.0, 0.0, g.s);
        n = 0;
        for (int k : g.alive) {
          Ctx& c = *g.c[k];
          c.layers[l].buf[sd].adj[SideNet::ROOT] = l < L ? P(c.rho[l + 1]) : P(c.rho[L]);
          ++n;
        }
        side_backward_n(net, bs, n, *g.ex, need_op, oo, 0.5, true, du, dw, 1.0, g.s);
      }
    });
    each(g, [&](int k) {
      Ctx& c = *g.c[k];
      if (need_op) herm(c, P(c.rho[l]), opn(c, c.layers[l].cf), g.s);
    });
  }
  // projection and |G_v|
  std::vector<char> finite(g.nb, 1);
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    Eval& E = *g.E[k];
    for (int i = 0; i < c.nt; ++i)
      project_tensor(c, i, g.W[k] + c.offs[i], P(E.D) + c.offs[i], P(E.G) + c.offs[i], g.s);
    E.delta.resize(c.nt);
    finite[k] = std::isfinite(E.e);
    for (int i = 0; i < c.nt; ++i) {
      const double* gi = P(E.G) + c.offs[i];
      E.delta[i] = std::sqrt(c.red.dot(gi, gi, c.rows[i] * c.cols[i] * c.rs, g.s));
      finite[k] = finite[k] && std::isfinite(E.delta[i]);
    }
  });
  check_group_flag(g);
  each(g, [&](int k) {
    Ctx& c = *g.c[k];
    Eval& E = *g.E[k];
    if (!finite[k]) throw Error(MERA_ERR_NONFINITE, "non-finite energy or gradient");
    compute_rho_v(c, E, g.W[k], g.s);
    E.eig_ready = false;
    E.valid = true;
  });
}

}  // namespace

void eval_group(Ctx* const* cs, const double* const* Ws, Eval* const* Es, int nb, bool grad, const Exec& ex,
                cudaStream_t s, std::exception_ptr* errs) {
  if (nb < 1 || nb > tc::TcEpilogue::MAXB) throw Error(MERA_ERR_ARG, "eval_group: member count out of range");
  Grp g;
  g.c = cs;
  g.W = Ws;
  g.E = Es;
  g.nb = nb;
  g.ex = &ex;
  g.s = s;
  g.err.assign(nb, nullptr);
  for (int k = 0; k < nb; ++k) {
    g.alive.push_back(k);
    cs[k]->prof.energy_grad_calls += grad ? 1 : 0;
    Es[k]->valid = false;
  }
  forward(g);
  if (grad) {
    series(g);
    reverse(g);
  }
  for (int k = 0; k < nb; ++k) errs[k] = g.err[k];
}

}  // namespace mera
