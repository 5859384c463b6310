// Host check of the contraction plans (mera::host_plan): the dense plan, its
// Z2 charge sectors and the real view of complex operands.  Built by
// tests/test_plan_host.py and linked against libmera.so; needs no GPU.
//
// For random pairwise contractions (2 to 4 legs per operand, extents 2 to 5,
// shared legs and output order drawn at random) of random Z2-symmetric
// tensors (entries of odd total charge zero), it applies every plan with a
// host loop of the GETT definition
//   C[cm[m] + cn[n]] = sum_k A[am[m] + ak[k]] B[bk[k] + bn[n]]  (+ beta C)
// and checks that
//   * the dense plan reproduces the definition (a sum over every assignment of
//     the legs);
//   * the two sector plans together reproduce the dense result entry by entry,
//     and the dense result is itself symmetric;
//   * the sectors write disjoint entries, exactly the entries of even charge;
//   * with every extent even, each sector holds 1/8 of the dense
//     multiply-adds (the pair 1/4);
//   * the output layout hints of every plan hold for its tables (c_rows: the
//     M offsets run contiguously through aligned groups of 32; c_vec = v: N
//     divisible by v, the N offsets run contiguously through aligned groups of
//     v, every M offset and every group-start N offset a multiple of v; and
//     the same for the transposed product).
// Then, for random complex contractions (interleaved storage, either operand
// conjugated, beta 0 or not), the four real products of mera::complex_parts on
// the real view (mera::real_view) reproduce alpha op(A) op(B) + beta C computed
// from the definition, and the real view's output hints hold.
// Finally the library's networks build on a dry table pool: the data-defined
// ternary and binary ones with charge-sector plans and real views, the sliced
// binary executor with real views.
// Prints "ok <cases>", "complex ok <cases>", "networks ok <n>" and the grading
// of extents 1..6 on success, else the first failure, and exits non-zero.
#include "tn.h"
#include "tnet.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

using mera::HostGroup;
using mera::HostPlan;
using mera::TDesc;

namespace {

TDesc desc(const std::vector<int>& legs, const std::vector<int64_t>& ext) {
  TDesc d;
  d.legs = legs;
  d.ext = ext;
  d.stride.assign(legs.size(), 1);
  for (size_t j = legs.size(); j-- > 1;) d.stride[j - 1] = d.stride[j] * ext[j];
  return d;
}

int64_t off(const HostGroup& g, int64_t i) { return g.table.empty() ? i * g.stride : g.table[i]; }

std::vector<int64_t> offsets(const HostGroup& g) {
  std::vector<int64_t> o(g.count);
  for (int64_t i = 0; i < g.count; ++i) o[i] = off(g, i);
  return o;
}

// total Z2 charge of storage index x of t
int charge(const TDesc& t, int64_t x) {
  int c = 0;
  for (size_t j = 0; j < t.legs.size(); ++j) c ^= mera::z2_charge((x / t.stride[j]) % t.ext[j], t.ext[j]);
  return c;
}

std::vector<double> symmetric_random(const TDesc& t, std::mt19937_64& rng) {
  std::normal_distribution<double> nd;
  std::vector<double> v(t.size());
  for (int64_t x = 0; x < t.size(); ++x) v[x] = charge(t, x) ? 0.0 : nd(rng);
  return v;
}

void apply(const HostPlan& h, const std::vector<double>& A, const std::vector<double>& B, std::vector<double>& C,
           std::vector<int>* touched) {
  for (int64_t m = 0; m < h.M; ++m)
    for (int64_t n = 0; n < h.N; ++n) {
      double s = 0.0;
      for (int64_t k = 0; k < h.K; ++k) s += A[off(h.am, m) + off(h.ak, k)] * B[off(h.bk, k) + off(h.bn, n)];
      const int64_t c = off(h.cm, m) + off(h.cn, n);
      C[c] = s;
      if (touched) (*touched)[c]++;
    }
}

bool runs_of(const std::vector<int64_t>& o, int64_t r) {
  for (size_t i = 0; i < o.size(); ++i)
    if (o[i] != o[i - i % r] + (int64_t)(i % r)) return false;
  return true;
}

bool vec_holds(const std::vector<int64_t>& rows, const std::vector<int64_t>& cols, int v) {
  if (v == 1) return true;
  if ((int64_t)cols.size() % v || !runs_of(cols, v)) return false;
  for (int64_t o : rows)
    if (o % v) return false;
  for (size_t i = 0; i < cols.size(); i += v)
    if (cols[i] % v) return false;
  return true;
}

bool hints_hold(const HostPlan& h) {
  const std::vector<int64_t> om = offsets(h.cm), on = offsets(h.cn);
  if (h.c_rows && !runs_of(om, 32)) return false;
  if (h.c_rows_t && !runs_of(on, 32)) return false;
  return vec_holds(om, on, h.c_vec) && vec_holds(on, om, h.c_vec_t);
}

}  // namespace

int main() {
  std::mt19937_64 rng(20200707);
  int cases = 0;
  for (int trial = 0; trial < 300; ++trial) {
    const bool even = trial % 3 == 0;  // every extent even: exact quarter of the work
    std::uniform_int_distribution<int> nlegs(1, 2), ext_d(2, 5), ext_e(1, 2);
    const int nm = nlegs(rng), nk = nlegs(rng), nn = nlegs(rng);
    // legs 0..nm-1 (M), nm..nm+nk-1 (K), then N
    std::vector<int64_t> ext(nm + nk + nn);
    for (auto& e : ext) e = even ? 2 * ext_e(rng) : ext_d(rng);
    std::vector<int> M, K, N;
    for (int i = 0; i < nm; ++i) M.push_back(i);
    for (int i = 0; i < nk; ++i) K.push_back(nm + i);
    for (int i = 0; i < nn; ++i) N.push_back(nm + nk + i);
    auto shuffled = [&](std::vector<int> v) {
      std::shuffle(v.begin(), v.end(), rng);
      return v;
    };
    auto exts = [&](const std::vector<int>& legs) {
      std::vector<int64_t> e;
      for (int l : legs) e.push_back(ext[l]);
      return e;
    };
    std::vector<int> la = M, lb = K, lc = M;
    la.insert(la.end(), K.begin(), K.end());
    lb.insert(lb.end(), N.begin(), N.end());
    lc.insert(lc.end(), N.begin(), N.end());
    la = shuffled(la);
    lb = shuffled(lb);
    lc = shuffled(lc);
    const TDesc A = desc(la, exts(la)), B = desc(lb, exts(lb)), C = desc(lc, exts(lc));
    const std::vector<double> a = symmetric_random(A, rng), b = symmetric_random(B, rng);
    const HostPlan hd = mera::host_plan(A, B, C, -1);
    std::vector<double> cd(C.size(), NAN), cs(C.size(), 0.0);
    std::vector<int> touched(C.size(), 0);
    apply(hd, a, b, cd, nullptr);
    // the dense plan against the definition: a sum over every assignment of the legs
    {
      const int nl = nm + nk + nn;
      std::vector<double> cref(C.size(), 0.0);
      std::vector<int64_t> idx(nl, 0);
      int64_t total = 1;
      for (int64_t e : ext) total *= e;
      auto at = [&](const TDesc& t) {
        int64_t o = 0;
        for (size_t j = 0; j < t.legs.size(); ++j) o += idx[t.legs[j]] * t.stride[j];
        return o;
      };
      for (int64_t i = 0; i < total; ++i) {
        cref[at(C)] += a[at(A)] * b[at(B)];
        for (int j = nl; j-- > 0;) {
          if (++idx[j] < ext[j]) break;
          idx[j] = 0;
        }
      }
      for (int64_t x = 0; x < C.size(); ++x)
        if (std::fabs(cref[x] - cd[x]) > 1e-13 * (1.0 + std::fabs(cref[x]))) {
          std::printf("trial %d: dense plan differs from the definition at %lld\n", trial, (long long)x);
          return 1;
        }
    }
    const HostPlan h0 = mera::host_plan(A, B, C, 0), h1 = mera::host_plan(A, B, C, 1);
    apply(h0, a, b, cs, &touched);
    apply(h1, a, b, cs, &touched);
    double scale = 1e-300;
    for (double x : cd) scale = std::max(scale, std::fabs(x));
    for (int64_t x = 0; x < C.size(); ++x) {
      const int want = charge(C, x) ? 0 : 1;
      if (touched[x] != want) {
        std::printf("trial %d: entry %lld written %d times (charge %d)\n", trial, (long long)x, touched[x],
                    charge(C, x));
        return 1;
      }
      if (charge(C, x) && cd[x] != 0.0) {
        std::printf("trial %d: dense result not symmetric at %lld\n", trial, (long long)x);
        return 1;
      }
      if (std::fabs(cd[x] - cs[x]) > 1e-13 * scale) {
        std::printf("trial %d: entry %lld dense %.17g sectors %.17g\n", trial, (long long)x, cd[x], cs[x]);
        return 1;
      }
    }
    if (even) {
      const int64_t dense = hd.M * hd.N * hd.K;
      if (8 * h0.M * h0.N * h0.K != dense || 8 * h1.M * h1.N * h1.K != dense) {
        std::printf("trial %d: sector work %lld + %lld of dense %lld\n", trial, (long long)(h0.M * h0.N * h0.K),
                    (long long)(h1.M * h1.N * h1.K), (long long)dense);
        return 1;
      }
    }
    for (const HostPlan* h : {&hd, &h0, &h1})
      if (!hints_hold(*h)) {
        std::printf("trial %d: an output layout hint does not hold\n", trial);
        return 1;
      }
    ++cases;
  }
  std::printf("ok %d\n", cases);
  // complex products through the real view
  int ccases = 0;
  for (int trial = 0; trial < 200; ++trial) {
    std::uniform_int_distribution<int> nlegs(1, 2), ext_d(1, 4), bit(0, 1);
    std::normal_distribution<double> nd;
    const int nm = nlegs(rng), nk = nlegs(rng), nn = nlegs(rng), nl = nm + nk + nn;
    std::vector<int64_t> ext(nl);
    for (auto& e : ext) e = ext_d(rng);
    std::vector<int> la, lb, lc;
    for (int i = 0; i < nm; ++i) { la.push_back(i); lc.push_back(i); }
    for (int i = nm; i < nm + nk; ++i) { la.push_back(i); lb.push_back(i); }
    for (int i = nm + nk; i < nl; ++i) { lb.push_back(i); lc.push_back(i); }
    std::shuffle(la.begin(), la.end(), rng);
    std::shuffle(lb.begin(), lb.end(), rng);
    std::shuffle(lc.begin(), lc.end(), rng);
    auto exts = [&](const std::vector<int>& legs) {
      std::vector<int64_t> e;
      for (int l : legs) e.push_back(ext[l]);
      return e;
    };
    const TDesc A = desc(la, exts(la)), B = desc(lb, exts(lb)), C = desc(lc, exts(lc));
    auto rnd = [&](int64_t n) {
      std::vector<double> v(2 * n);
      for (double& x : v) x = nd(rng);
      return v;
    };
    const std::vector<double> a = rnd(A.size()), b = rnd(B.size()), c0 = rnd(C.size());
    const bool ac = bit(rng), bc = bit(rng);
    const double alpha = nd(rng), beta = bit(rng) ? 0.0 : nd(rng);
    // definition: complex sum over every assignment of the legs
    std::vector<double> cref(2 * C.size(), 0.0);
    {
      std::vector<int64_t> idx(nl, 0);
      int64_t total = 1;
      for (int64_t e : ext) total *= e;
      auto at = [&](const TDesc& t) {
        int64_t o = 0;
        for (size_t j = 0; j < t.legs.size(); ++j) o += idx[t.legs[j]] * t.stride[j];
        return o;
      };
      for (int64_t i = 0; i < total; ++i) {
        const int64_t ia = at(A), ib = at(B), ic = at(C);
        const double ar = a[2 * ia], ai = ac ? -a[2 * ia + 1] : a[2 * ia + 1];
        const double br = b[2 * ib], bi = bc ? -b[2 * ib + 1] : b[2 * ib + 1];
        cref[2 * ic] += ar * br - ai * bi;
        cref[2 * ic + 1] += ar * bi + ai * br;
        for (int j = nl; j-- > 0;) {
          if (++idx[j] < ext[j]) break;
          idx[j] = 0;
        }
      }
      for (int64_t x = 0; x < 2 * C.size(); ++x) cref[x] = alpha * cref[x] + beta * c0[x];
    }
    // the four real products on the real view, with the GETT's alpha/beta rule
    const HostPlan r = mera::real_view(mera::host_plan(A, B, C, -1));
    std::vector<double> cs = c0;
    for (const mera::ComplexPart& pt : mera::complex_parts(ac, bc)) {
      const double al = pt.sign * alpha, be = pt.first ? beta : 1.0;
      for (int64_t m = 0; m < r.M; ++m)
        for (int64_t n = 0; n < r.N; ++n) {
          double sum = 0.0;
          for (int64_t k = 0; k < r.K; ++k)
            sum += a[pt.ca + off(r.am, m) + off(r.ak, k)] * b[pt.cb + off(r.bk, k) + off(r.bn, n)];
          double& dst = cs[pt.cc + off(r.cm, m) + off(r.cn, n)];
          dst = be != 0.0 ? be * dst + al * sum : al * sum;
        }
    }
    for (int64_t x = 0; x < 2 * C.size(); ++x)
      if (std::fabs(cs[x] - cref[x]) > 1e-12 * (1.0 + std::fabs(cref[x]))) {
        std::printf("complex trial %d: entry %lld real view %.17g definition %.17g\n", trial, (long long)x, cs[x],
                    cref[x]);
        return 1;
      }
    if (!hints_hold(r)) {
      std::printf("complex trial %d: an output layout hint of the real view does not hold\n", trial);
      return 1;
    }
    ++ccases;
  }
  std::printf("complex ok %d\n", ccases);
  // the library's own networks build in every mode (dry table pool: no device)
  int nets = 0;
  try {
    for (const std::array<int64_t, 2> dims :
         {std::array<int64_t, 2>{2, 8}, std::array<int64_t, 2>{8, 8}, std::array<int64_t, 2>{4, 16}}) {
      for (int mode = 0; mode < 3; ++mode) {  // 0 dense, 1 Z2 sectors, 2 real views (complex, mixed)
        mera::TablePool pool(true);
        pool.set_real_view(mode == 2);
        for (char side : {'L', 'C', 'R'}) {
          mera::Net net(mera::ternary_netdef(side), dims[0], dims[1], pool, mode == 1);
          for (const mera::GemmPlan* p : net.plans())
            if (mode == 2 && !p->proto.has_rv) throw std::runtime_error("a ternary plan without its real view");
          ++nets;
        }
        for (char side : {'L', 'R'}) {  // the binary network as data (Z2 binary problems)
          mera::Net net(mera::binary_netdef(side), dims[0], dims[1], pool, mode == 1);
          for (const mera::GemmPlan* p : net.plans())
            if (mode == 2 && !p->proto.has_rv) throw std::runtime_error("a binary plan without its real view");
          ++nets;
        }
        if (mode != 1)
          for (char side : {'L', 'R'}) {
            mera::SideNet net(side, dims[0], dims[1], pool, dims[1] / 2);
            for (const mera::GemmPlan* p : net.executed_plans())
              if (mode == 2 && !p->proto.has_rv) throw std::runtime_error("a binary plan without its real view");
            ++nets;
          }
      }
    }
  } catch (const std::exception& e) {
    std::printf("networks: %s\n", e.what());
    return 1;
  }
  std::printf("networks ok %d\n", nets);
  // the grading, for comparison with the input generators
  for (int64_t e = 1; e <= 6; ++e) {
    std::printf("grading %lld:", (long long)e);
    for (int64_t i = 0; i < e; ++i) std::printf(" %d", mera::z2_charge(i, e));
    std::printf("\n");
  }
  return 0;
}
