// The C ABI of include/mera.h: argument checks, error codes, copies in and
// out of the caller's arrays, the footprint dry runs, counters.
#include "ctx.h"

#include <cmath>
#include <cstring>
#include <mutex>

namespace mera {
namespace {
std::mutex g_alloc_mu;
Allocator g_alloc;
}  // namespace
Allocator current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc;
}
}  // namespace mera

// ================================================================ C ABI ====
using mera::Error;

namespace {
struct Guard {
  mera_t m;
  explicit Guard(mera_t mm) : m(mm) { mera::g_prof = mm ? &mm->prof : nullptr; }
  ~Guard() { mera::g_prof = nullptr; }
};

// After a failed call: if a tensor-core wait expired during it, that is the
// cause (an aborted product leaves garbage that later steps may report as
// non-convergence or non-finite values), so the flag is cleared and the
// error reported as MERA_ERR_DEVICE_TIMEOUT.  The Krylov warm starts are
// invalid then too.
bool take_device_flag(mera_t m) {
  if (!m || !m->tc_err.p) return false;
  int e = 0;
  if (cudaMemcpyAsync(&e, m->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, m->s) != cudaSuccess ||
      cudaStreamSynchronize(m->s) != cudaSuccess)
    return false;
  if (!e) return false;
  (void)cudaMemsetAsync(m->tc_err.p, 0, sizeof(int), m->s);
  m->have_rho = m->have_x = false;
  return true;
}

template <class F>
int wrap(mera_t m, F&& f) {
  Guard g(m);
  try {
    f();
    return MERA_OK;
  } catch (const Error& e) {
    if (e.code != MERA_ERR_DEVICE_TIMEOUT && take_device_flag(m)) {
      m->err = std::string("a bounded tensor-core wait expired (then: ") + e.what() + ")";
      return MERA_ERR_DEVICE_TIMEOUT;
    }
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
// A step with a NaN or infinite entry has a non-finite squared norm.
void check_finite_step(mera_t m, const double* X) {
  const double q = m->red.dot(X, X, m->total, m->s);
  if (!std::isfinite(q)) throw Error(MERA_ERR_NONFINITE, "the step has a non-finite entry");
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
  c->device_wait_s = 1.0;
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
      if (m->z2) {
        std::vector<int64_t> rows, cols;
        mera::tensor_legs(*m, i, rows, cols);
        rq = mera::fused_charges(rows);
        cq = mera::fused_charges(cols);
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
  if (!m || !X || !Y || !std::isfinite(alpha)) return MERA_ERR_ARG;
  return wrap(m, [&] {
    copy_in(m, X, mera::P(m->dir2));
    check_finite_step(m, mera::P(m->dir2));
    copy_in(m, (const void* const*)Y, mera::P(m->tmpv));
    mera::make_geom(*m, mera::P(m->Wcur), mera::P(m->dir2), alpha, m->s);
    mera::apply_transport(*m, mera::P(m->Wcur), mera::P(m->dir2), mera::P(m->tmpv), m->s);
    copy_out(m, mera::P(m->tmpv), Y);
  });
}

int mera_retract(mera_t m, const void* const* X, double alpha, void* const* Xprime) {
  if (!m || !X || !std::isfinite(alpha)) return MERA_ERR_ARG;
  return wrap(m, [&] {
    copy_in(m, X, mera::P(m->dir2));
    check_finite_step(m, mera::P(m->dir2));
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

int mera_gd_step(mera_t m, mera_iter_info* info) {
  if (!m || !info) return MERA_ERR_ARG;
  return wrap(m, [&] { mera::gd_step(*m, info, m->s); });
}

int mera_ev_sweep(mera_t m, double gamma, mera_iter_info* info) {
  if (!m || !info || !std::isfinite(gamma)) return MERA_ERR_ARG;
  return wrap(m, [&] {
    std::memset(info, 0, sizeof(*info));
    mera::ev_sweep(*m, gamma, info, m->s);
  });
}

int mera_solve(mera_t m, const mera_solve_opts* o, mera_solve_result* r) {
  if (!m || !o || !r || o->method < 0 || o->method > 2 || o->maxiter < 0) return MERA_ERR_ARG;
  return wrap(m, [&] {
    std::memset(r, 0, sizeof(*r));
    mera::ensure_current(*m, m->s);
    mera_iter_info info{};
    double gn = std::sqrt(mera::inner(*m, mera::P(m->ev[m->cur].G), mera::P(m->ev[m->cur].G), m->s));
    r->n_evals = 1;
    for (int it = 0; it < o->maxiter && !(gn < o->gtol); ++it) {
      if (o->method == 1) mera::cg_step(*m, &info, m->s);
      else if (o->method == 2) mera::gd_step(*m, &info, m->s);
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
// mera_footprint_bytes for the data-defined networks: the ternary MERA, or
// the binary one with Z2 charge sectors (0 where its chain would be sliced)
size_t footprint_net(const mera_config* cfg) {
  const bool tern = cfg->network == MERA_TERNARY;
  const int ns = tern ? 2 : 3;  // sites of a level operator
  std::vector<int64_t> dims{cfg->d_b};
  for (int l = 0; l < cfg->n_trans; ++l) {
    const int64_t d = dims.back();
    dims.push_back(std::min<int64_t>(cfg->chi, tern ? d * d * d : d * d));
  }
  if (dims.back() != cfg->chi) return 0;
  const bool mixed = cfg->prec != MERA_PREC_FP64;
  const size_t rs = cfg->dtype == MERA_C128 ? 2 : 1;
  const size_t es = (mixed ? 4 : 8) * rs;
  mera::TablePool pool(true);
  size_t bytes = 0, ws = 0, total = 0, gmax = 1;
  for (size_t l = 0; l < dims.size(); ++l) {
    const int64_t cf = dims[l], cc = l + 1 < dims.size() ? dims[l + 1] : dims[l];
    if (!tern && (mera::choose_chunk(cf, cc) != 0 || (cfg->b_chunk > 0 && cfg->b_chunk < cc))) return 0;
    const int64_t wr = tern ? cf * cf * cf : cf * cf;
    total += (cf * cf * cf * cf + wr * cc) * rs;
    bytes += 2 * 8 * rs * (size_t)mera::ipow(cf, 2 * ns);  // h_l, rho_l
    gmax = std::max<size_t>({gmax, (size_t)(cf * cf * cf * cf), (size_t)(cc * cc * cc * cc),
                             (size_t)(cf * cf * cc * cc * cc), (size_t)(cf * cc * cc * cf),
                             (size_t)(cf * cc * cf * cf * cf)});
    if (tern)
      gmax = std::max<size_t>({gmax, (size_t)(cf * cf * cf * cc), (size_t)(cf * cf * cf * cc * cc * cc),
                               (size_t)(cf * cf * cf * cf * cf * cc)});
    for (char sd : std::string(tern ? "LCR" : "LR")) {
      mera::Net net(tern ? mera::ternary_netdef(sd) : mera::binary_netdef(sd), cf, cc, pool, cfg->z2 == 1);
      for (int node = net.nleaf(); node < net.nnode(); ++node)
        bytes += es * (size_t)net.size(node) * (node == net.root() ? 1 : 2);
      for (const mera::GemmPlan* p : net.plans()) ws = std::max(ws, mera::tc_workspace_bytes(p->proto, cfg->prec));
    }
  }
  const size_t nS = (size_t)mera::ipow(cfg->chi, 2 * ns) * rs;
  bytes += ws + pool.bytes();
  bytes += 8 * nS * (size_t)(std::max(2, cfg->krylov_dim) + 1 + 3);  // basis, tmp, x, bvec
  bytes += 8 * gmax * 6 * rs * rs;
  bytes += 8 * (size_t)total * (size_t)(2 * std::max(1, cfg->lbfgs_m) + 2 + 4 + 4);
  return bytes;
}
}  // namespace

size_t mera_footprint_bytes(const mera_config* cfg) {
  if (!cfg || !mera::config_range_error(*cfg).empty()) return 0;
  if (cfg->dtype != MERA_F64 && cfg->dtype != MERA_C128) return 0;
  if (cfg->prec < MERA_PREC_FP64 || cfg->prec > MERA_PREC_SPLIT_FP16) return 0;
  if (cfg->z2 != 0 && (cfg->z2 != 1 || cfg->network == MERA_MPS)) return 0;
  if (cfg->network == MERA_MPS) return footprint_mps(cfg);
  if (cfg->d_b < 2 || cfg->chi < 2 || cfg->n_trans < 1) return 0;
  if (cfg->network == MERA_TERNARY || (cfg->network == MERA_BINARY && cfg->z2 == 1)) {
    try {
      return footprint_net(cfg);
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

int mera_reset_warm_starts(mera_t m) {
  if (!m) return MERA_ERR_ARG;
  m->have_rho = m->have_x = false;
  return MERA_OK;
}

int mera_set_device_wait(mera_t m, double seconds) {
  if (!m || !(seconds > 0.0 && seconds <= 60.0)) return MERA_ERR_ARG;
  m->cfg.device_wait_s = seconds;
  m->ex.wait_ns = (uint64_t)(seconds * 1e9);
  return MERA_OK;
}

int mera_set_allocator(mera_alloc_fn alloc, mera_free_fn dealloc, void* user) {
  if (alloc && !dealloc) return MERA_ERR_ARG;
  std::lock_guard<std::mutex> lk(mera::g_alloc_mu);
  mera::g_alloc.alloc = alloc;
  mera::g_alloc.dealloc = alloc ? dealloc : nullptr;
  mera::g_alloc.user = alloc ? user : nullptr;
  return MERA_OK;
}

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
    if (prec != MERA_PREC_3XTF32 && prec != MERA_PREC_SPLIT_BF16 && prec != MERA_PREC_SPLIT_FP16)
      throw Error(MERA_ERR_ARG, "bad precision");
    const int kind = mera::tc::kind_of_prec(prec);
    const int elem = mera::tc::kind_elem(kind);
    const int64_t Kp = mera::tc::padded_k(K, kind);
    const int64_t Mp = mera::tc::round_up(std::max<int64_t>(M, 1), 128), Np = mera::tc::round_up(std::max<int64_t>(N, 1), 128);
    mera::DevBuf ah(elem * Mp * Kp), al(elem * Mp * Kp), bh(elem * Np * Kp), bl(elem * Np * Kp), err(sizeof(int));
    const size_t skb = mera::tc::splitk_bytes(M, N, Kp, kind);
    mera::DevBuf part(skb), amax(2 * sizeof(unsigned)), ctr(sizeof(unsigned long long));
    unsigned* am = amax.as<unsigned>();
    MERA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    mera::tc::pack_split(A, true, nullptr, K, nullptr, 1, M, K, Mp, Kp, kind, ah.p, al.p, false, s, am);
    mera::tc::pack_split(B, true, nullptr, 1, nullptr, N, N, K, Np, Kp, kind, bh.p, bl.p, true, s, am + 1);
    mera::tc::TcEpilogue ep;
    if (kind == mera::tc::KIND_F16) {
      ep.a_amax = am;
      ep.b_amax = am + 1;
    }
    ep.C = C;
    ep.c_f64 = 1;
    ep.cms = N;
    ep.cns = 1;
    ep.rows = N == 1;
    ep.err = err.as<int>();
    ep.work_ctr = ctr.as<unsigned long long>();
    mera::tc::gemm_packed(kind, M, N, Kp, ah.p, al.p, Mp, bh.p, bl.p, Np, ep, s, part.as<float>(), skb);
    int e = 0;
    MERA_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MERA_CUDA(cudaStreamSynchronize(s));
    if (e) throw Error(MERA_ERR_DEVICE_TIMEOUT, "tensor-core GEMM: a bounded wait expired");
  });
}

}  // extern "C"
