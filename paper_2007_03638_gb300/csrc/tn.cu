// Contraction trees of the binary MERA ascending maps and their reverse-mode
// (adjoint) passes.
//
// A_L(o) (operator on fine sites 0,1,2) and A_R(o) (fine sites 1,2,3) are
// 11-tensor networks (Sec. 4; standard binary MERA).  Both are evaluated
// with the same binary tree, found by an exhaustive search over pairwise
// orders: 2.125 chi^9 multiply-adds with two chi^9 steps and one 7-leg
// intermediate (N5), which no later step needs to keep.
//
// The scalar s = Tr(A(o) rho) is differentiated in reverse mode through the
// tree: the root adjoint is rho, the adjoint of the operator leaf is the
// descending map D(rho), and the adjoints of the conjugated u/w copies are
// the environments whose sum is the partial derivative D_v (Sec. 4).  One
// forward plus one reverse pass cost 5.3 chi^9 per side instead of
// 15 chi^9 for separate ascending, descending and ten environment networks.
#include "tn.h"
#include "tc_gemm.h"
#include <algorithm>
#include <cstring>

namespace mera {

const int64_t* TablePool::get(const std::vector<int64_t>& host) {
  if (dry_) {
    bytes_ += sizeof(int64_t) * host.size();
    static int64_t dummy = 0;
    return &dummy;
  }
  auto it = tables_.find(host);
  if (it != tables_.end()) return it->second.as<int64_t>();
  DevBuf buf(sizeof(int64_t) * host.size());
  MERA_CUDA(cudaMemcpyAsync(buf.p, host.data(), sizeof(int64_t) * host.size(), cudaMemcpyHostToDevice, stream_));
  MERA_CUDA(cudaStreamSynchronize(stream_));
  bytes_ += buf.bytes;
  const int64_t* p = buf.as<int64_t>();
  tables_.emplace(host, std::move(buf));
  return p;
}

namespace {
// Offsets of every multi-index of a leg group (row-major over the group).
// Returns false (and sets *stride) if the group is affine, i.e. offset = i * stride.
bool group_offsets(const std::vector<int64_t>& ext, const std::vector<int64_t>& str,
                   std::vector<int64_t>& out, int64_t* stride) {
  int64_t n = 1;
  for (auto e : ext) n *= e;
  std::vector<int64_t> e2, s2;
  for (size_t j = 0; j < ext.size(); ++j)
    if (ext[j] > 1) { e2.push_back(ext[j]); s2.push_back(str[j]); }
  if (e2.empty()) { *stride = 0; return false; }
  bool affine = true;
  for (size_t j = 0; j + 1 < e2.size(); ++j)
    if (s2[j] != s2[j + 1] * e2[j + 1]) affine = false;
  if (affine) { *stride = s2.back(); return false; }
  out.assign(n, 0);
  std::vector<int64_t> idx(ext.size(), 0);
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i) {
    out[i] = o;
    for (size_t j = ext.size(); j-- > 0;) {
      if (++idx[j] < ext[j]) { o += str[j]; break; }
      o -= str[j] * (ext[j] - 1);
      idx[j] = 0;
    }
  }
  return true;
}

// off(i) = off(i - i % r) + i % r for every i
bool runs_of(const std::vector<int64_t>& off, int64_t r) {
  for (size_t i = 0; i < off.size(); ++i)
    if (off[i] != off[i - i % r] + (int64_t)(i % r)) return false;
  return true;
}

TDesc make_desc(const std::vector<int>& legs, const std::vector<int64_t>& ext) {
  TDesc d;
  d.legs = legs;
  d.ext = ext;
  d.stride.assign(legs.size(), 1);
  for (size_t j = legs.size(); j-- > 1;) d.stride[j - 1] = d.stride[j] * ext[j];
  return d;
}
}  // namespace

std::vector<int64_t> sector_offsets(const TDesc& t, const std::vector<int>& legs, int q) {
  std::vector<int64_t> ext, str;
  int64_t n = 1;
  for (int l : legs) {
    const int j = t.find(l);
    if (j < 0) throw Error(MERA_ERR_ARG, "sector_offsets: leg not in the tensor");
    ext.push_back(t.ext[j]);
    str.push_back(t.stride[j]);
    n *= t.ext[j];
  }
  std::vector<int64_t> out;
  out.reserve(q < 0 ? n : n / 2 + 1);
  std::vector<int64_t> idx(ext.size(), 0);
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i) {
    int ch = 0;
    for (size_t j = 0; j < ext.size(); ++j) ch ^= z2_charge(idx[j], ext[j]);
    if (q < 0 || ch == q) out.push_back(o);
    for (size_t j = ext.size(); j-- > 0;) {
      if (++idx[j] < ext[j]) { o += str[j]; break; }
      o -= str[j] * (ext[j] - 1);
      idx[j] = 0;
    }
  }
  return out;
}

namespace {
// Dense group: a table, or an affine stride (the tables the dense path has
// always used).
HostGroup dense_group(const TDesc& t, const std::vector<int>& legs) {
  std::vector<int64_t> ext, str;
  HostGroup g;
  g.count = 1;
  for (int l : legs) {
    const int j = t.find(l);
    ext.push_back(t.ext[j]);
    str.push_back(t.stride[j]);
    g.count *= t.ext[j];
  }
  int64_t s = 0;
  if (!group_offsets(ext, str, g.table, &s)) {
    g.table.clear();
    g.stride = s;
  }
  return g;
}

HostGroup sector_group(const TDesc& t, const std::vector<int>& legs, int q) {
  HostGroup g;
  g.table = sector_offsets(t, legs, q);
  g.count = (int64_t)g.table.size();
  return g;
}

std::vector<int64_t> offsets_of(const HostGroup& g) {
  if (!g.table.empty()) return g.table;
  std::vector<int64_t> o(g.count);
  for (int64_t i = 0; i < g.count; ++i) o[i] = i * g.stride;
  return o;
}

HostGroup doubled(const HostGroup& g) {
  HostGroup r = g;
  for (int64_t& o : r.table) o *= 2;
  r.stride *= 2;
  return r;
}

// Output layout hints (see GettCall) of the M-group and N-group offsets of C,
// for C = A B and for C^T = B^T A^T.
void set_hints(HostPlan& h, const std::vector<int64_t>& om, const std::vector<int64_t>& on) {
  auto vec_of = [](const std::vector<int64_t>& rows, const std::vector<int64_t>& cols) {
    for (int64_t v : {8, 4}) {
      if ((int64_t)cols.size() % v || !runs_of(cols, v)) continue;
      bool ok = true;
      for (int64_t o : rows) ok = ok && o % v == 0;
      for (size_t i = 0; i < cols.size() && ok; i += v) ok = cols[i] % v == 0;
      if (ok) return (int)v;
    }
    return 1;
  };
  h.c_rows = runs_of(om, 32);
  h.c_vec = vec_of(om, on);
  h.c_rows_t = runs_of(on, 32);
  h.c_vec_t = vec_of(on, om);
}

const int64_t* upload(const HostGroup& g, TablePool& pool, int64_t* stride) {
  if (g.table.empty()) {
    *stride = g.stride;
    return nullptr;
  }
  *stride = 0;
  return pool.get(g.table);
}
}  // namespace

HostPlan host_plan(const TDesc& A, const TDesc& B, const TDesc& C, int q) {
  std::vector<int> M, N, K;
  for (int l : C.legs) {
    const bool inA = A.find(l) >= 0, inB = B.find(l) >= 0;
    if (inA == inB) throw Error(MERA_ERR_ARG, "make_plan: output leg in both/neither operand");
    (inA ? M : N).push_back(l);
  }
  for (int l : B.legs)
    if (C.find(l) < 0) {
      if (A.find(l) < 0) throw Error(MERA_ERR_ARG, "make_plan: dangling leg in B");
      K.push_back(l);
    }
  for (int l : A.legs)
    if (C.find(l) < 0 && B.find(l) < 0) throw Error(MERA_ERR_ARG, "make_plan: dangling leg in A");
  // where is each operand's stride-1 leg?
  auto fast_leg = [](const TDesc& t) {
    int best = -1;
    for (size_t j = 0; j < t.legs.size(); ++j)
      if (t.ext[j] > 1 && (best < 0 || t.stride[j] < t.stride[best])) best = (int)j;
    return best < 0 ? -1 : t.legs[best];
  };
  const int fa = fast_leg(A), fb = fast_leg(B);
  {
    // K is summed, so its enumeration order is free (both operands' tables
    // follow it): the larger operand whose stride-1 leg is summed gets that
    // leg innermost, so that its packing reads consecutive k along memory
    const bool fa_k = std::find(K.begin(), K.end(), fa) != K.end();
    const bool fb_k = std::find(K.begin(), K.end(), fb) != K.end();
    const int pick = fa_k && fb_k ? (A.size() >= B.size() ? fa : fb) : fa_k ? fa : fb_k ? fb : -1;
    if (pick >= 0) {
      K.erase(std::find(K.begin(), K.end(), pick));
      K.push_back(pick);
    }
  }
  HostPlan h;
  auto grp = [&](const TDesc& t, const std::vector<int>& legs) {
    return q < 0 ? dense_group(t, legs) : sector_group(t, legs, q);
  };
  h.am = grp(A, M);
  h.ak = grp(A, K);
  h.bk = grp(B, K);
  h.bn = grp(B, N);
  h.cm = grp(C, M);
  h.cn = grp(C, N);
  if (h.am.count != h.cm.count || h.bn.count != h.cn.count || h.ak.count != h.bk.count)
    throw Error(MERA_ERR_ARG, "make_plan: extent mismatch");
  h.M = h.am.count;
  h.N = h.bn.count;
  h.K = h.ak.count;
  if (q >= 0 && h.M > 0 && h.N > 0 && h.K == 0)
    throw Error(MERA_ERR_UNSUPPORTED, "make_plan: a charge sector with outputs but no summed index");
  // orientation hints for operand packing
  h.a_rfast = std::find(M.begin(), M.end(), fa) != M.end();
  h.b_rfast = std::find(N.begin(), N.end(), fb) != N.end();
  set_hints(h, offsets_of(h.cm), offsets_of(h.cn));
  return h;
}

HostPlan real_view(const HostPlan& h) {
  HostPlan r = h;
  for (HostGroup* g : {&r.am, &r.ak, &r.bk, &r.bn, &r.cm, &r.cn}) *g = doubled(*g);
  set_hints(r, offsets_of(r.cm), offsets_of(r.cn));
  return r;
}

std::array<ComplexPart, 4> complex_parts(bool a_conj, bool b_conj) {
  auto sign = [&](int ca, int cb) {
    double sg = ca && cb ? -1.0 : 1.0;  // i * i = -1
    if (ca && a_conj) sg = -sg;
    if (cb && b_conj) sg = -sg;
    return sg;
  };
  return {{{0, 0, 0, sign(0, 0), true},
           {1, 1, 0, sign(1, 1), false},
           {0, 1, 1, sign(0, 1), true},
           {1, 0, 1, sign(1, 0), false}}};
}

GemmPlan upload_plan(const HostPlan& h, TablePool& pool) {
  GemmPlan p;
  GettCall& g = p.proto;
  g.a.t0 = upload(h.am, pool, &g.a.s0);
  g.a.t1 = upload(h.ak, pool, &g.a.s1);
  g.b.t0 = upload(h.bk, pool, &g.b.s0);
  g.b.t1 = upload(h.bn, pool, &g.b.s1);
  g.c.t0 = upload(h.cm, pool, &g.c.s0);
  g.c.t1 = upload(h.cn, pool, &g.c.s1);
  g.M = h.M;
  g.N = h.N;
  g.K = h.K;
  g.a_rfast = h.a_rfast;
  g.b_rfast = h.b_rfast;
  g.c_rows = h.c_rows;
  g.c_vec = h.c_vec;
  g.c_rows_t = h.c_rows_t;
  g.c_vec_t = h.c_vec_t;
  if (pool.real_view()) {
    const HostPlan r = real_view(h);
    g.ar.t0 = upload(r.am, pool, &g.ar.s0);
    g.ar.t1 = upload(r.ak, pool, &g.ar.s1);
    g.br.t0 = upload(r.bk, pool, &g.br.s0);
    g.br.t1 = upload(r.bn, pool, &g.br.s1);
    g.cr.t0 = upload(r.cm, pool, &g.cr.s0);
    g.cr.t1 = upload(r.cn, pool, &g.cr.s1);
    g.cr_rows = r.c_rows;
    g.cr_vec = r.c_vec;
    g.cr_rows_t = r.c_rows_t;
    g.cr_vec_t = r.c_vec_t;
    g.has_rv = 1;
  }
  return p;
}

GemmPlan make_plan(const TDesc& A, const TDesc& B, const TDesc& C, TablePool& pool, int q) {
  return upload_plan(host_plan(A, B, C, q), pool);
}

// N1..N10 children (node ids).
const int SideNet::kids_[10][2] = {
    {7, 8},    // N1 = conj w_far  x w_far
    {0, 1},    // N2 = o x conj u_in
    {12, 2},   // N3 = N2 x u_in
    {3, 4},    // N4 = conj u_half x conj w_mid
    {13, 14},  // N5 = N3 x N4            (7 legs)
    {5, 6},    // N6 = u_half x w_mid
    {15, 16},  // N7 = N5 x N6
    {11, 17},  // N8 = N1 x N7
    {9, 10},   // N9 = conj w_near x w_near
    {18, 19},  // N10 = N8 x N9 = ascended operator
};

SideNet::SideNet(char side, int64_t cf, int64_t cc, TablePool& pool, int64_t chunk) : side_(side) {
  // leg names -> ids; coarse legs a b c (conj side) A B C (plain side)
  std::map<std::string, int> id;
  auto L = [&](const char* names) {  // split on spaces (re-entrant: objects are built concurrently)
    std::vector<int> v;
    std::string cur;
    for (const char* p = names;; ++p) {
      if (*p == ' ' || *p == 0) {
        if (!cur.empty()) {
          auto it = id.find(cur);
          if (it == id.end()) it = id.emplace(cur, (int)id.size()).first;
          v.push_back(it->second);
          cur.clear();
        }
        if (*p == 0) break;
      } else {
        cur += *p;
      }
    }
    return v;
  };
  const char* names[NLEAF];
  if (side == 'L') {
    const char* n[NLEAF] = {"f0 f1 f2 g0 g1 g2", "f1 f2 x1 x2", "g1 g2 y1 y2", "fm f0 xm x0",
                            "x0 x1 b",           "fm g0 ym y0", "y0 y1 B",     "xl xm a",
                            "xl ym A",           "x2 x3 c",     "y2 x3 C"};
    std::copy(n, n + NLEAF, names);
  } else {
    const char* n[NLEAF] = {"f1 f2 f3 g1 g2 g3", "f1 f2 x1 x2", "g1 g2 y1 y2", "f3 f4 x3 x4",
                            "x2 x3 b",           "g3 f4 y3 y4", "y2 y3 B",     "x4 x5 c",
                            "y4 x5 C",           "x0 x1 a",     "x0 y1 A"};
    std::copy(n, n + NLEAF, names);
  }
  const std::vector<int> coarse = L("a b c A B C");
  auto extent = [&](int leg) {
    return std::find(coarse.begin(), coarse.end(), leg) != coarse.end() ? cc : cf;
  };
  for (int i = 0; i < NLEAF; ++i) {
    auto legs = L(names[i]);
    std::vector<int64_t> ext;
    for (int l : legs) ext.push_back(extent(l));
    desc_[i] = make_desc(legs, ext);
  }
  // internal nodes: free legs of the left child (its order) then of the right child
  std::vector<int> count(64, 0);
  for (int i = 0; i < NLEAF; ++i)
    for (int l : desc_[i].legs) count[l]++;
  for (int k = 0; k < 10; ++k) {
    const TDesc& a = desc_[kids_[k][0]];
    const TDesc& b = desc_[kids_[k][1]];
    std::vector<int> legs;
    std::vector<int64_t> ext;
    for (size_t j = 0; j < a.legs.size(); ++j)
      if (b.find(a.legs[j]) < 0) { legs.push_back(a.legs[j]); ext.push_back(a.ext[j]); }
    for (size_t j = 0; j < b.legs.size(); ++j)
      if (a.find(b.legs[j]) < 0) { legs.push_back(b.legs[j]); ext.push_back(b.ext[j]); }
    if (NLEAF + k == ROOT) {
      // root: [a b c A B C]
      std::vector<int64_t> e6(6, cc);
      desc_[ROOT] = make_desc(coarse, e6);
      if (legs.size() != 6) throw Error(MERA_ERR_ARG, "SideNet: root legs");
    } else {
      desc_[NLEAF + k] = make_desc(legs, ext);
    }
  }
  for (int k = 0; k < 10; ++k) {
    const int node = NLEAF + k, l = kids_[k][0], r = kids_[k][1];
    fwd_[k] = make_plan(desc_[l], desc_[r], desc_[node], pool);
    TDesc dnode = desc_[node];
    if (node == ROOT) {
      // root adjoint is rho with memory layout [A B C a b c]
      dnode = make_desc(L("A B C a b c"), std::vector<int64_t>(6, cc));
    }
    TDesc dl = desc_[l];
    if (l == 0) {
      // adjoint of the operator leaf is written as the descended operator,
      // i.e. transposed: rows = plain-side fine legs, columns = conj-side legs
      std::vector<int> legs(dl.legs.begin() + 3, dl.legs.end());
      legs.insert(legs.end(), dl.legs.begin(), dl.legs.begin() + 3);
      dl = make_desc(legs, std::vector<int64_t>(6, cf));
    }
    bwdl_[k] = make_plan(dnode, desc_[r], dl, pool);
    bwdr_[k] = make_plan(desc_[l], dnode, desc_[r], pool);
  }
  cc_ = cc;
  if (chunk > 0 && chunk < cc) {
    if (cc % chunk) throw Error(MERA_ERR_ARG, "SideNet: chunk must divide the coarse dimension");
    sliced_ = true;
    nb_ = chunk;
    const int b = id.at("b");
    auto view = [&](const TDesc& d) {  // same strides, leg b restricted to one slice
      TDesc v = d;
      v.ext[d.find(b)] = chunk;
      return v;
    };
    const TDesc& n3 = desc_[13];
    const TDesc& n4 = desc_[14];
    const TDesc& n6 = desc_[16];
    const TDesc& n7 = desc_[17];
    std::vector<int64_t> e5 = desc_[15].ext;
    e5[desc_[15].find(b)] = chunk;
    n5c_ = make_desc(desc_[15].legs, e5);
    sb4_ = n4.stride[n4.find(b)];
    sb7_ = n7.stride[n7.find(b)];
    f5c_ = make_plan(n3, view(n4), n5c_, pool);
    f7c_ = make_plan(n5c_, n6, view(n7), pool);
    b7c_ = make_plan(view(n7), n6, n5c_, pool);
    b5lc_ = make_plan(n5c_, view(n4), n3, pool);
    b5rc_ = make_plan(n3, n5c_, view(n4), pool);
  }
}

std::vector<const GemmPlan*> SideNet::executed_plans() const {
  std::vector<const GemmPlan*> v;
  for (int node = NLEAF; node < NNODE; ++node) {
    if (sliced_ && (node == 15 || node == 17)) {
      // only the sliced chi^9 chain runs; N7's other child (N6) gets no adjoint
      continue;
    }
    v.push_back(&fwd(node));
    v.push_back(&bwd_left(node));
    v.push_back(&bwd_right(node));
  }
  if (sliced_) {
    for (const GemmPlan* p : {&f5c_, &f7c_, &b7c_, &b5lc_, &b5rc_}) v.push_back(p);
  }
  return v;
}

double SideNet::forward_flops() const {
  double f = 0;
  for (auto& p : fwd_) f += p.flops();
  return f;
}

// Workspace of one tensor-core product of nb members: two words per member
// for the operands' maxima (FP16 planes), the members' four planes, the
// split-K partials; 1024-byte aligned regions.
size_t tc_workspace_bytes(const GettCall& g, int prec, int nb) {
  if (prec == MERA_PREC_FP64) return 0;
  const int kind = tc::kind_of_prec(prec);
  const size_t elem = tc::kind_elem(kind);
  const int64_t Kp = tc::padded_k(g.K, kind);
  const int64_t Mp = tc::round_up(g.M, 128), Np = tc::round_up(g.N, 128);
  return 6 * 1024 + (size_t)nb * (elem * 2 * (size_t)(Mp + Np) * (size_t)Kp + tc::splitk_bytes(g.M, g.N, Kp, kind));
}

// A keep slot: the operand's maximum word, then its two planes.
size_t tc_keep_bytes(const GettCall& g, int prec, int side) {
  if (prec == MERA_PREC_FP64 || side == 0) return 0;
  const int kind = tc::kind_of_prec(prec);
  const size_t elem = tc::kind_elem(kind);
  const int64_t Kp = tc::padded_k(g.K, kind);
  const int64_t Rp = tc::round_up(side == 1 ? g.M : g.N, 128);
  return 3 * 1024 + elem * 2 * (size_t)Rp * (size_t)Kp;
}

void keep_need(const SideNet& net, int prec, size_t need[2]) {
  need[0] = need[1] = 0;
  if (!net.sliced()) return;
  need[0] = std::max(tc_keep_bytes(net.f5c().proto, prec, 1), tc_keep_bytes(net.b5rc().proto, prec, 1));
  need[1] = std::max(tc_keep_bytes(net.f7c().proto, prec, 2), tc_keep_bytes(net.b7c().proto, prec, 2));
}

namespace {
// The transposed product C^T = B^T A^T: the same contraction with the roles
// of A and B (and of the M and N groups) exchanged.
GettCall transposed(const GettCall& g) {
  GettCall h = g;
  h.A = g.B;
  h.B = g.A;
  h.a.t0 = g.b.t1; h.a.s0 = g.b.s1;  // rows of A^T-side operand: B's N group
  h.a.t1 = g.b.t0; h.a.s1 = g.b.s0;  // its K group
  h.b.t0 = g.a.t1; h.b.s0 = g.a.s1;  // K group of the other: A's K group
  h.b.t1 = g.a.t0; h.b.s1 = g.a.s0;  // its N group: A's M group
  h.c.t0 = g.c.t1; h.c.s0 = g.c.s1;
  h.c.t1 = g.c.t0; h.c.s1 = g.c.s0;
  h.M = g.N;
  h.N = g.M;
  h.a32 = g.b32;
  h.b32 = g.a32;
  h.a_conj = g.b_conj;
  h.b_conj = g.a_conj;
  h.a_rfast = g.b_rfast;
  h.b_rfast = g.a_rfast;
  h.c_rows = g.c_rows_t;
  h.c_vec = g.c_vec_t;
  h.c_rows_t = g.c_rows;
  h.c_vec_t = g.c_vec;
  h.a_amax = g.b_amax;
  h.b_amax = g.a_amax;
  return h;
}
}  // namespace

void contract(const GettCall& g0, const Exec& ex, cudaStream_t s, const Keep* keep) {
  if (g0.M <= 0 || g0.N <= 0) return;
  if (ex.prec == MERA_PREC_FP64) {
    if (g0.a32 || g0.b32 || g0.c32) throw Error(MERA_ERR_ARG, "contract: float operand in the FP64 path");
    gett_f64(g0, s);
    return;
  }
  if (g0.cplx) {
    // complex operands: four real products of the real views (no keep slot:
    // every part packs its own components)
    if (!g0.has_rv) throw Error(MERA_ERR_UNSUPPORTED, "contract: complex tensor-core product without a real view");
    auto part_ptr = [](const double* p, bool f32, int comp) {
      return f32 ? reinterpret_cast<const double*>(reinterpret_cast<const float*>(p) + comp) : p + comp;
    };
    // the output's maximum covers both components: begun once for all parts
    const bool track = g0.c_amax && ex.prec == MERA_PREC_SPLIT_FP16;
    if (track && g0.beta == 0.0 && !g0.c_amax_started) MERA_CUDA(cudaMemsetAsync(g0.c_amax, 0, sizeof(unsigned), s));
    for (const ComplexPart& pt : complex_parts(g0.a_conj != 0, g0.b_conj != 0)) {
      GettCall h = g0;
      h.cplx = h.a_conj = h.b_conj = h.has_rv = 0;
      h.a = g0.ar;
      h.b = g0.br;
      h.c = g0.cr;
      h.c_rows = g0.cr_rows;
      h.c_vec = g0.cr_vec;
      h.c_rows_t = g0.cr_rows_t;
      h.c_vec_t = g0.cr_vec_t;
      h.A = part_ptr(g0.A, g0.a32, pt.ca);
      h.B = part_ptr(g0.B, g0.b32, pt.cb);
      h.C = const_cast<double*>(part_ptr(g0.C, g0.c32, pt.cc));
      h.alpha = pt.sign * g0.alpha;
      h.beta = pt.first ? g0.beta : 1.0;
      h.c_amax_started = 1;
      contract(h, ex, s, nullptr);
    }
    return;
  }
  // tensor cores: take the orientation whose output columns run contiguously
  // (the epilogue then writes whole 32-byte pieces of each row)
  const bool flip = g0.c_vec < 8 && g0.c_vec_t > g0.c_vec;
  const GettCall g = flip ? transposed(g0) : g0;
  int kside = keep ? keep->side : 0;  // kept operand, as a side of g
  if (flip && kside) kside = 3 - kside;
  const int kind = tc::kind_of_prec(ex.prec);
  const size_t elem = tc::kind_elem(kind);
  const int64_t Kp = tc::padded_k(g.K, kind);
  const int64_t Mp = tc::round_up(g.M, 128), Np = tc::round_up(g.N, 128);
  if (tc_workspace_bytes(g, ex.prec) > ex.ws_bytes) throw Error(MERA_ERR_ARG, "contract: workspace too small");
  auto align = [](size_t o) { return (o + 1023) & ~size_t(1023); };
  char* w = static_cast<char*>(ex.ws);
  unsigned* amax_a = reinterpret_cast<unsigned*>(w);  // maxima of the operands (FP16 planes)
  unsigned* amax_b = amax_a + 1;
  // byte 128: the product's work-item counter
  size_t o = 1024;
  void* ah = w + o; o = align(o + elem * Mp * Kp);
  void* al = w + o; o = align(o + elem * Mp * Kp);
  void* bh = w + o; o = align(o + elem * Np * Kp);
  void* bl = w + o; o = align(o + elem * Np * Kp);
  float* part = reinterpret_cast<float*>(w + o);
  const size_t part_bytes = ex.ws_bytes > o ? ex.ws_bytes - o : 0;
  if (kside) {
    // the kept operand's planes live in their slot
    const int slot = keep->slot;
    if (slot < 0 || slot > 1 || !ex.keep[slot] || ex.keep_bytes[slot] < tc_keep_bytes(g, ex.prec, kside))
      throw Error(MERA_ERR_ARG, "contract: keep slot missing or too small");
    char* k = static_cast<char*>(ex.keep[slot]);
    const int64_t Rp = kside == 1 ? Mp : Np;
    (kside == 1 ? amax_a : amax_b) = reinterpret_cast<unsigned*>(k);
    (kside == 1 ? ah : bh) = k + 1024;
    (kside == 1 ? al : bl) = k + 1024 + align(elem * Rp * Kp);
  }
  const bool pack_a = !(kside == 1 && keep->valid), pack_b = !(kside == 2 && keep->valid);
  // FP16 planes: an operand's maximum known from its producer is used as it
  // is (no reduction pass); a kept operand carries its maximum in its slot
  const unsigned* known_a = nullptr;
  const unsigned* known_b = nullptr;
  if (kind == tc::KIND_F16) {
    if (g.a_amax) {
      if (kside == 1) {
        if (pack_a) MERA_CUDA(cudaMemcpyAsync(amax_a, g.a_amax, sizeof(unsigned), cudaMemcpyDeviceToDevice, s));
      } else {
        known_a = g.a_amax;
      }
    }
    if (g.b_amax) {
      if (kside == 2) {
        if (pack_b) MERA_CUDA(cudaMemcpyAsync(amax_b, g.b_amax, sizeof(unsigned), cudaMemcpyDeviceToDevice, s));
      } else {
        known_b = g.b_amax;
      }
    }
  }
  const bool copied_a = kind == tc::KIND_F16 && g.a_amax && kside == 1;  // slot word already holds it
  const bool copied_b = kind == tc::KIND_F16 && g.b_amax && kside == 2;
  // A rows = M group, A columns = K group; B rows (of the packed K-major plane) = N group
  Prof* pr = g_prof;
  int64_t pair = -1;
  if (pack_a) {
    pair = pr ? pr->begin(g.M, g.K, 0, s) : -1;
    tc::pack_split(g.A, !g.a32, g.a.t0, g.a.s0, g.a.t1, g.a.s1, g.M, g.K, Mp, Kp, kind, ah, al, g.a_rfast, s,
                   amax_a, known_a ? known_a : (copied_a ? amax_a : nullptr));
    if (pr) pr->end(pair, 9100 + (g.a_rfast ? 10 : 0) + (g.a32 ? 1 : 0), s);
  }
  if (pack_b) {
    pair = pr ? pr->begin(g.N, g.K, 0, s) : -1;
    tc::pack_split(g.B, !g.b32, g.b.t1, g.b.s1, g.b.t0, g.b.s0, g.N, g.K, Np, Kp, kind, bh, bl, g.b_rfast, s,
                   amax_b, known_b ? known_b : (copied_b ? amax_b : nullptr));
    if (pr) pr->end(pair, 9200 + (g.b_rfast ? 10 : 0) + (g.b32 ? 1 : 0), s);
  }
  tc::TcEpilogue ep;
  ep.alpha = g.alpha;
  ep.beta = g.beta;
  ep.cm = g.c.t0;
  ep.cms = g.c.s0;
  ep.cn = g.c.t1;
  ep.cns = g.c.s1;
  ep.C = g.C;
  ep.c_f64 = g.c32 ? 0 : 1;
  ep.rows = g.c_rows;
  ep.vec = g.c_vec;
  ep.err = ex.err;
  ep.wait_ns = ex.wait_ns;
  ep.work_ctr = reinterpret_cast<unsigned long long*>(w + 128);
  if (kind == tc::KIND_F16) {
    ep.a_amax = known_a ? known_a : amax_a;
    ep.b_amax = known_b ? known_b : amax_b;
    if (g.c_amax) {
      if (g.beta == 0.0 && !g.c_amax_started) MERA_CUDA(cudaMemsetAsync(g.c_amax, 0, sizeof(unsigned), s));
      ep.c_amax = g.c_amax;
    }
  }
  pair = pr ? pr->begin(g.M, g.N, g.K, s) : -1;
  const int path = tc::gemm_packed(kind, g.M, g.N, Kp, ah, al, Mp, bh, bl, Np, ep, s, part, part_bytes);
  if (pr) {
    pr->end(pair, 1000 * (kind + 1) + 100 * path, s);
    pr->gett_launches++;
    pr->gett_flops += 2.0 * (double)g.M * (double)g.N * (double)g.K;
  }
}

void contract_batch(const GettCall* gs, int nb, const Exec& ex, cudaStream_t s) {
  if (nb == 1) {
    contract(gs[0], ex, s, nullptr);
    return;
  }
  const GettCall& g0 = gs[0];
  if (g0.M <= 0 || g0.N <= 0) return;
  if (nb > tc::TcEpilogue::MAXB) throw Error(MERA_ERR_ARG, "contract_batch: too many members");
  if (ex.prec == MERA_PREC_FP64 || g0.cplx) {
    // FP64 and complex products run member by member
    for (int b = 0; b < nb; ++b) contract(gs[b], ex, s, nullptr);
    return;
  }
  // one tensor-core launch for every member: the same orientation and plan
  // (tables of member 0: the members' tables are equal by construction)
  const bool flip = g0.c_vec < 8 && g0.c_vec_t > g0.c_vec;
  const int kind = tc::kind_of_prec(ex.prec);
  const size_t elem = tc::kind_elem(kind);
  GettCall g[tc::TcEpilogue::MAXB];
  for (int b = 0; b < nb; ++b) g[b] = flip ? transposed(gs[b]) : gs[b];
  const GettCall& h = g[0];
  const int64_t Kp = tc::padded_k(h.K, kind);
  const int64_t Mp = tc::round_up(h.M, 128), Np = tc::round_up(h.N, 128);
  if (tc_workspace_bytes(h, ex.prec, nb) > ex.ws_bytes) throw Error(MERA_ERR_ARG, "contract_batch: workspace too small");
  auto align = [](size_t o) { return (o + 1023) & ~size_t(1023); };
  char* w = static_cast<char*>(ex.ws);
  unsigned* amax = reinterpret_cast<unsigned*>(w);  // member b: words 2b (A), 2b + 1 (B); byte 128: work counter
  size_t o = 1024;
  char* ah = w + o; o = align(o + elem * nb * Mp * Kp);
  char* al = w + o; o = align(o + elem * nb * Mp * Kp);
  char* bh = w + o; o = align(o + elem * nb * Np * Kp);
  char* bl = w + o; o = align(o + elem * nb * Np * Kp);
  float* part = reinterpret_cast<float*>(w + o);
  const size_t part_bytes = ex.ws_bytes > o ? ex.ws_bytes - o : 0;
  tc::TcEpilogue ep;
  ep.nb = nb;
  Prof* pr = g_prof;
  for (int b = 0; b < nb; ++b) {
    const GettCall& x = g[b];
    const bool f16 = kind == tc::KIND_F16;
    int64_t pair = pr ? pr->begin(x.M, x.K, 0, s) : -1;
    tc::pack_split(x.A, !x.a32, h.a.t0, h.a.s0, h.a.t1, h.a.s1, x.M, x.K, Mp, Kp, kind, ah + elem * b * Mp * Kp,
                   al + elem * b * Mp * Kp, x.a_rfast, s, amax + 2 * b, f16 ? x.a_amax : nullptr);
    if (pr) pr->end(pair, 9100 + (x.a_rfast ? 10 : 0) + (x.a32 ? 1 : 0), s);
    pair = pr ? pr->begin(x.N, x.K, 0, s) : -1;
    tc::pack_split(x.B, !x.b32, h.b.t1, h.b.s1, h.b.t0, h.b.s0, x.N, x.K, Np, Kp, kind, bh + elem * b * Np * Kp,
                   bl + elem * b * Np * Kp, x.b_rfast, s, amax + 2 * b + 1, f16 ? x.b_amax : nullptr);
    if (pr) pr->end(pair, 9200 + (x.b_rfast ? 10 : 0) + (x.b32 ? 1 : 0), s);
    ep.member_C[b] = x.C;
    if (f16) {
      ep.member_amax_a[b] = x.a_amax ? x.a_amax : amax + 2 * b;
      ep.member_amax_b[b] = x.b_amax ? x.b_amax : amax + 2 * b + 1;
      if (x.c_amax) {
        if (x.beta == 0.0 && !x.c_amax_started) MERA_CUDA(cudaMemsetAsync(x.c_amax, 0, sizeof(unsigned), s));
        ep.member_cmax[b] = x.c_amax;
      }
    }
  }
  ep.C = g[0].C;
  ep.alpha = h.alpha;
  ep.beta = h.beta;
  ep.cm = h.c.t0;
  ep.cms = h.c.s0;
  ep.cn = h.c.t1;
  ep.cns = h.c.s1;
  ep.c_f64 = h.c32 ? 0 : 1;
  ep.rows = h.c_rows;
  ep.vec = h.c_vec;
  ep.err = ex.err;
  ep.wait_ns = ex.wait_ns;
  ep.work_ctr = reinterpret_cast<unsigned long long*>(w + 128);
  const int64_t pair = pr ? pr->begin(h.M, h.N, h.K, s) : -1;
  const int path = tc::gemm_packed(kind, h.M, h.N, Kp, ah, al, Mp, bh, bl, Np, ep, s, part, part_bytes);
  if (pr) {
    pr->end(pair, 1000 * (kind + 1) + 100 * path, s);
    pr->gett_launches++;
    pr->gett_flops += 2.0 * (double)h.M * (double)h.N * (double)h.K * nb;
  }
}

namespace {
inline bool internal(int node) { return node >= SideNet::NLEAF && node != SideNet::ROOT; }
// conjugated copies of u and w (bra side of <MERA| ... |MERA>)
inline bool conj_leaf(int node) { return node == 1 || node == 3 || node == 4 || node == 7 || node == 9; }
constexpr int EXT = -1;  // an external buffer (operator, seed, output): double, never conjugated

// Run one plan.  Operands are identified by node id (or EXT): leaves and
// externals are double, internal nodes float in mixed mode; conjugated
// leaves are read conjugated.
// Operands of one member's product: pointers and maximum words (see
// SideBufs::amax); cstart: the output's maximum was begun by an earlier
// slice of the same buffer.
struct Ops {
  const double* A = nullptr;
  const double* B = nullptr;
  double* C = nullptr;
  const unsigned* aa = nullptr;
  const unsigned* ba = nullptr;
  unsigned* ca = nullptr;
  int cstart = 0;
};

// Run one plan for every member; ops(b, k) gives member k's operands.
// Operands are identified by node id (or EXT): leaves and externals are
// double, internal nodes float in mixed mode; conjugated leaves are read
// conjugated.  One member: the product may keep an operand's planes.
template <class F>
void run_n(SideBufs* const* bs, int nb, const Exec& ex, const GemmPlan& p, int an, int bn, int cn, double alpha,
           double beta, cudaStream_t s, const Keep* keep, F ops) {
  GettCall g[tc::TcEpilogue::MAXB];
  for (int k = 0; k < nb; ++k) {
    const SideBufs& b = *bs[k];
    const Ops o = ops(b, k);
    GettCall& x = g[k];
    x = p.proto;
    x.A = o.A;
    x.B = o.B;
    x.C = o.C;
    x.a_amax = o.aa;
    x.b_amax = o.ba;
    x.c_amax = o.ca;
    x.c_amax_started = o.cstart;
    x.alpha = alpha;
    x.beta = beta;
    x.a32 = b.f32 && an != EXT && internal(an);
    x.b32 = b.f32 && bn != EXT && internal(bn);
    x.c32 = b.f32 && cn != EXT && internal(cn);
    x.cplx = b.cplx;
    x.a_conj = b.cplx && an != EXT && conj_leaf(an);
    x.b_conj = b.cplx && bn != EXT && conj_leaf(bn);
  }
  if (nb == 1)
    contract(g[0], ex, s, keep);
  else
    contract_batch(g, nb, ex, s);
}
inline const double* value(const SideBufs& b, int node) {
  return node < SideNet::NLEAF ? b.leaf[node] : b.val[node];
}
// maximum words of an internal node's value and adjoint (null for leaves,
// the root and when the buffers carry none)
inline unsigned* vmax(const SideBufs& b, int node) {
  return b.amax && internal(node) ? b.amax + node : nullptr;
}
inline unsigned* amax_adj(const SideBufs& b, int node) {
  return b.amax && internal(node) ? b.amax + SideNet::NNODE + node : nullptr;
}
// Advance a node pointer by `off` elements of its storage type.
inline double* offp(const SideBufs& b, const double* p, int64_t off) {
  char* c = reinterpret_cast<char*>(const_cast<double*>(p));
  return reinterpret_cast<double*>(c + off * (b.f32 ? 4 : 8) * (b.cplx ? 2 : 1));
}
}  // namespace

void side_prepare_n(const SideNet& net, SideBufs* const* bs, int nb, const Exec& ex, cudaStream_t s) {
  for (int node : {11, 14, 16, 19}) {
    const int l = SideNet::left(node), r = SideNet::right(node);
    run_n(bs, nb, ex, net.fwd(node), l, r, node, 1.0, 0.0, s, nullptr, [&](const SideBufs& b, int) {
      return Ops{value(b, l), value(b, r), b.val[node], vmax(b, l), vmax(b, r), vmax(b, node)};
    });
  }
}

void side_forward_n(const SideNet& net, SideBufs* const* bs, int nb, const Exec& ex, double* const* out,
                    double alpha, double beta, cudaStream_t s) {
  if (net.sliced() && nb > 1) throw Error(MERA_ERR_UNSUPPORTED, "side_forward: a sliced chain runs one member at a time");
  for (int node : {12, 13, 15, 17, 18}) {
    if (net.sliced() && node == 15) {
      // N5 = N3 x N4 and N7 = N5 x N6 one slice of the coarse leg b at a time
      // N3 and N6 are the same for every slice: their packed planes are kept
      for (int64_t b0 = 0; b0 < net.coarse(); b0 += net.chunk()) {
        const Keep k3{1, 0, b0 > 0}, k6{2, 1, b0 > 0};
        run_n(bs, 1, ex, net.f5c(), 13, 14, 15, 1.0, 0.0, s, ex.keep[0] ? &k3 : nullptr,
              [&](const SideBufs& b, int) {
                return Ops{b.val[13], offp(b, b.val[14], b0 * net.b_stride_n4()), b.val[15], vmax(b, 13),
                           vmax(b, 14), vmax(b, 15)};
              });
        run_n(bs, 1, ex, net.f7c(), 15, 16, 17, 1.0, 0.0, s, ex.keep[1] ? &k6 : nullptr,
              [&](const SideBufs& b, int) {
                return Ops{b.val[15], b.val[16], offp(b, b.val[17], b0 * net.b_stride_n7()), vmax(b, 15),
                           vmax(b, 16), vmax(b, 17), b0 > 0};
              });
      }
      continue;
    }
    if (net.sliced() && node == 17) continue;
    const int l = SideNet::left(node), r = SideNet::right(node);
    run_n(bs, nb, ex, net.fwd(node), l, r, node, 1.0, 0.0, s, nullptr, [&](const SideBufs& b, int) {
      return Ops{value(b, l), value(b, r), b.val[node], vmax(b, l), vmax(b, r), vmax(b, node)};
    });
  }
  if (out)
    run_n(bs, nb, ex, net.fwd(SideNet::ROOT), 18, 19, EXT, alpha, beta, s, nullptr, [&](const SideBufs& b, int k) {
      return Ops{b.val[18], b.val[19], out[k], vmax(b, 18), vmax(b, 19)};
    });
}

void side_backward_n(const SideNet& net, SideBufs* const* bs, int nb, const Exec& ex, bool need_op,
                     double* const* op_out, double alpha_op, bool need_env, double* const* du, double* const* dw,
                     double alpha_env, cudaStream_t s) {
  if (net.sliced() && nb > 1) throw Error(MERA_ERR_UNSUPPORTED, "side_backward: a sliced chain runs one member at a time");
  // which nodes need an adjoint: subtree contains the operator (need_op) or a
  // conjugated u/w leaf (need_env)
  bool need[SideNet::NNODE] = {};
  if (need_op) need[0] = true;
  if (need_env)
    for (int l : {1, 3, 4, 7, 9}) need[l] = true;
  for (int node = SideNet::NLEAF; node < SideNet::NNODE; ++node)
    need[node] = need[SideNet::left(node)] || need[SideNet::right(node)];
  for (int node = SideNet::ROOT; node >= SideNet::NLEAF; --node) {
    if (!need[node]) continue;
    if (net.sliced() && node == 15) continue;  // handled with N7 below
    if (net.sliced() && node == 17) {
      // dN5 one slice of b at a time, consumed at once by N5's children
      // N6 and N3 are the same for every slice: their packed planes are kept
      for (int64_t b0 = 0; b0 < net.coarse(); b0 += net.chunk()) {
        const Keep k6{2, 1, b0 > 0}, k3{1, 0, b0 > 0};
        run_n(bs, 1, ex, net.b7c(), 17, 16, 15, 1.0, 0.0, s, ex.keep[1] ? &k6 : nullptr,
              [&](const SideBufs& b, int) {
                return Ops{offp(b, b.adj[17], b0 * net.b_stride_n7()), b.val[16], b.adj[15], amax_adj(b, 17),
                           vmax(b, 16), amax_adj(b, 15)};
              });
        if (need[13])
          run_n(bs, 1, ex, net.b5lc(), 15, 14, 13, 1.0, b0 == 0 ? 0.0 : 1.0, s, nullptr,
                [&](const SideBufs& b, int) {
                  return Ops{b.adj[15], offp(b, b.val[14], b0 * net.b_stride_n4()), b.adj[13], amax_adj(b, 15),
                             vmax(b, 14), amax_adj(b, 13)};
                });
        if (need[14])
          run_n(bs, 1, ex, net.b5rc(), 13, 15, 14, 1.0, 0.0, s, ex.keep[0] ? &k3 : nullptr,
                [&](const SideBufs& b, int) {
                  return Ops{b.val[13], b.adj[15], offp(b, b.adj[14], b0 * net.b_stride_n4()), vmax(b, 13),
                             amax_adj(b, 15), amax_adj(b, 14), b0 > 0};
                });
      }
      continue;
    }
    const int l = SideNet::left(node), r = SideNet::right(node);
    for (int side = 0; side < 2; ++side) {
      const int c = side == 0 ? l : r;
      if (!need[c]) continue;
      double alpha = 1.0, beta = 0.0;
      if (c == 0) {
        alpha = alpha_op; beta = 1.0;
      } else if (c < SideNet::NLEAF) {
        alpha = alpha_env; beta = 1.0;
      }
      auto out_of = [&](const SideBufs& b, int k) -> double* {
        if (c == 0) return op_out[k];
        if (c < SideNet::NLEAF) return (c == 1 || c == 3) ? du[k] : dw[k];
        return b.adj[c];
      };
      // the adjoint of node is internal (node id) unless node is the root (seed rho: external);
      // a leaf's adjoint goes to an external accumulator
      const int dn_id = node != SideNet::ROOT ? node : EXT;
      const int out_id = c >= SideNet::NLEAF ? c : EXT;
      if (side == 0)
        run_n(bs, nb, ex, net.bwd_left(node), dn_id, r, out_id, alpha, beta, s, nullptr,
              [&](const SideBufs& b, int k) {
                return Ops{b.adj[node], value(b, r), out_of(b, k), amax_adj(b, node), vmax(b, r),
                           c >= SideNet::NLEAF ? amax_adj(b, c) : nullptr};
              });
      else
        run_n(bs, nb, ex, net.bwd_right(node), l, dn_id, out_id, alpha, beta, s, nullptr,
              [&](const SideBufs& b, int k) {
                return Ops{value(b, l), b.adj[node], out_of(b, k), vmax(b, l), amax_adj(b, node),
                           c >= SideNet::NLEAF ? amax_adj(b, c) : nullptr};
              });
    }
  }
}

void side_prepare(const SideNet& net, SideBufs& b, cudaStream_t s) {
  SideBufs* bs[1] = {&b};
  side_prepare_n(net, bs, 1, *b.ex, s);
}

void side_forward(const SideNet& net, SideBufs& b, double* out, double alpha, double beta, cudaStream_t s) {
  SideBufs* bs[1] = {&b};
  double* o[1] = {out};
  side_forward_n(net, bs, 1, *b.ex, out ? o : nullptr, alpha, beta, s);
}

void side_backward(const SideNet& net, SideBufs& b, bool need_op, double* op_out, double alpha_op,
                   bool need_env, double* du, double* dw, double alpha_env, cudaStream_t s) {
  SideBufs* bs[1] = {&b};
  double* oo[1] = {op_out};
  double* u[1] = {du};
  double* w[1] = {dw};
  side_backward_n(net, bs, 1, *b.ex, need_op, oo, alpha_op, need_env, u, w, alpha_env, s);
}

}  // namespace mera
