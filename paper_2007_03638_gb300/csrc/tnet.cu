// Tensor network given as data (see tnet.h) and the ternary MERA networks.
#include "tnet.h"

#include <map>
#include <sstream>

namespace mera {

NetDef ternary_netdef(char side) {
  // Leaves: the operator on fine sites (f bra, g ket), then the conjugated and
  // plain copies of u and w in the cone; x legs join conjugated copies, y legs
  // plain ones, p/q legs are traced between a conjugated and a plain w.
  // Trees: the cheapest pairwise orders (exhaustive search; 2.13 chi^8 for
  // A_L and A_R, 0.02 chi^8 for A_C, no intermediate above chi^6).
  NetDef d;
  d.out = "a b A B";
  d.rho = "A B a b";
  d.op_adj = "g0 g1 f0 f1";
  if (side == 'L') {
    // o on fine (3j, 3j+1): u on (3j-1, 3j), w_{j-1} and w_j
    d.legs = {"f0 f1 g0 g1", "fm f0 xm x0", "p1 p2 xm a", "x0 f1 q2 b", "fm g0 ym y0", "p1 p2 ym A", "y0 g1 q2 B"};
    d.role = {ROLE_OP, ROLE_UB, ROLE_WB, ROLE_WB, ROLE_U, ROLE_W, ROLE_W};
    d.kids = {{0, 1}, {7, 3}, {8, 4}, {9, 6}, {2, 5}, {11, 10}};
  } else if (side == 'C') {
    // o on fine (3j+2, 3j+3): both sites under u, w_j and w_{j+1}
    d.legs = {"f0 f1 g0 g1", "f0 f1 x2 x3", "p0 p1 x2 a", "x3 p4 p5 b", "g0 g1 y2 y3", "p0 p1 y2 A", "y3 p4 p5 B"};
    d.role = {ROLE_OP, ROLE_UB, ROLE_WB, ROLE_WB, ROLE_U, ROLE_W, ROLE_W};
    d.kids = {{0, 1}, {7, 4}, {2, 5}, {8, 9}, {3, 6}, {10, 11}};
  } else if (side == 'R') {
    // o on fine (3j+1, 3j+2): site 3j+1 under no u, u on (3j+2, 3j+3)
    d.legs = {"f0 f1 g0 g1", "p0 f0 x2 a", "f1 fp x2 x3", "x3 p4 p5 b", "p0 g0 y2 A", "g1 fp y2 y3", "y3 p4 p5 B"};
    d.role = {ROLE_OP, ROLE_WB, ROLE_UB, ROLE_WB, ROLE_W, ROLE_U, ROLE_W};
    d.kids = {{0, 1}, {7, 2}, {8, 4}, {9, 5}, {3, 6}, {10, 11}};
  } else {
    throw Error(MERA_ERR_ARG, "ternary_netdef: side must be L, C or R");
  }
  return d;
}

NetDef binary_netdef(char side) {
  // The binary MERA's A_L (o on fine 0,1,2) and A_R (o on fine 1,2,3): the
  // same leaves, legs and pairwise tree as the sliced executor of tn.cu
  // (2.13 chi^9 per side, one 7-leg intermediate), given as data.
  NetDef d;
  d.out = "a b c A B C";
  d.rho = "A B C a b c";
  if (side == 'L') {
    d.legs = {"f0 f1 f2 g0 g1 g2", "f1 f2 x1 x2", "g1 g2 y1 y2", "fm f0 xm x0", "x0 x1 b", "fm g0 ym y0",
              "y0 y1 B", "xl xm a", "xl ym A", "x2 x3 c", "y2 x3 C"};
    d.op_adj = "g0 g1 g2 f0 f1 f2";
  } else if (side == 'R') {
    d.legs = {"f1 f2 f3 g1 g2 g3", "f1 f2 x1 x2", "g1 g2 y1 y2", "f3 f4 x3 x4", "x2 x3 b", "g3 f4 y3 y4",
              "y2 y3 B", "x4 x5 c", "y4 x5 C", "x0 x1 a", "x0 y1 A"};
    d.op_adj = "g1 g2 g3 f1 f2 f3";
  } else {
    throw Error(MERA_ERR_ARG, "binary_netdef: side must be L or R");
  }
  d.role = {ROLE_OP, ROLE_UB, ROLE_U, ROLE_UB, ROLE_WB, ROLE_U, ROLE_W, ROLE_WB, ROLE_W, ROLE_WB, ROLE_W};
  d.kids = {{7, 8}, {0, 1}, {12, 2}, {3, 4}, {13, 14}, {5, 6}, {15, 16}, {11, 17}, {9, 10}, {18, 19}};
  return d;
}

namespace {
std::vector<std::string> words(const std::string& s) {
  std::istringstream is(s);
  std::vector<std::string> out;
  std::string w;
  while (is >> w) out.push_back(w);
  return out;
}

TDesc desc_of(const std::vector<int>& legs, const std::vector<int64_t>& ext) {
  TDesc d;
  d.legs = legs;
  d.ext = ext;
  d.stride.assign(legs.size(), 1);
  for (size_t j = legs.size(); j-- > 1;) d.stride[j - 1] = d.stride[j] * ext[j];
  return d;
}

// The dense plan of a product, or its nonempty Z2 charge sectors.
PlanSet plans_of(const TDesc& A, const TDesc& B, const TDesc& C, TablePool& pool, bool z2) {
  PlanSet ps;
  if (!z2) {
    ps.p[0] = make_plan(A, B, C, pool);
    ps.n = 1;
    return ps;
  }
  for (int q = 0; q < 2; ++q) {
    const HostPlan h = host_plan(A, B, C, q);
    if (h.M > 0 && h.N > 0) ps.p[ps.n++] = upload_plan(h, pool);
  }
  return ps;
}
}  // namespace

Net::Net(const NetDef& d, int64_t cf, int64_t cc, TablePool& pool, bool z2) {
  nleaf_ = (int)d.legs.size();
  nnode_ = nleaf_ + (int)d.kids.size();
  kids_ = d.kids;
  role_ = d.role;
  if ((int)role_.size() != nleaf_ || nleaf_ < 2 || role_[0] != ROLE_OP)
    throw Error(MERA_ERR_ARG, "Net: leaf 0 must be the operator");
  std::map<std::string, int> id;
  std::vector<int64_t> ext_of_id;
  auto legs_of = [&](const std::string& s, std::vector<int64_t>& ext) {
    std::vector<int> out;
    ext.clear();
    for (const std::string& w : words(s)) {
      auto it = id.find(w);
      if (it == id.end()) {
        it = id.emplace(w, (int)id.size()).first;
        const bool coarse = w == "a" || w == "b" || w == "c" || w == "A" || w == "B" || w == "C";
        ext_of_id.push_back(coarse ? cc : cf);
      }
      out.push_back(it->second);
      ext.push_back(ext_of_id[it->second]);
    }
    return out;
  };
  desc_.resize(nnode_);
  fixed_.assign(nnode_, false);
  std::vector<int64_t> ext;
  for (int i = 0; i < nleaf_; ++i) {
    const std::vector<int> legs = legs_of(d.legs[i], ext);
    desc_[i] = desc_of(legs, ext);
    fixed_[i] = i != 0;
  }
  for (int k = 0; k < (int)kids_.size(); ++k) {
    const int node = nleaf_ + k, l = kids_[k][0], r = kids_[k][1];
    if (l < 0 || r < 0 || l >= node || r >= node) throw Error(MERA_ERR_ARG, "Net: children must precede a node");
    const TDesc &a = desc_[l], &b = desc_[r];
    std::vector<int> legs;
    std::vector<int64_t> e;
    for (size_t j = 0; j < a.legs.size(); ++j)
      if (b.find(a.legs[j]) < 0) { legs.push_back(a.legs[j]); e.push_back(a.ext[j]); }
    for (size_t j = 0; j < b.legs.size(); ++j)
      if (a.find(b.legs[j]) < 0) { legs.push_back(b.legs[j]); e.push_back(b.ext[j]); }
    desc_[node] = desc_of(legs, e);
    fixed_[node] = fixed_[l] && fixed_[r];
  }
  // the root is stored in the order of `out`
  const std::vector<int> out = legs_of(d.out, ext);
  if (out.size() != desc_[root()].legs.size()) throw Error(MERA_ERR_ARG, "Net: root legs differ from out");
  for (int leg : out)
    if (desc_[root()].find(leg) < 0) throw Error(MERA_ERR_ARG, "Net: root legs differ from out");
  desc_[root()] = desc_of(out, ext);
  std::vector<int64_t> e2;
  const TDesc seed = desc_of(legs_of(d.rho, e2), e2);
  const TDesc opadj = desc_of(legs_of(d.op_adj, e2), e2);
  for (int k = 0; k < (int)kids_.size(); ++k) {
    const int node = nleaf_ + k, l = kids_[k][0], r = kids_[k][1];
    fwd_.push_back(plans_of(desc_[l], desc_[r], desc_[node], pool, z2));
    const TDesc& dn = node == root() ? seed : desc_[node];
    bwdl_.push_back(plans_of(dn, desc_[r], l == 0 ? opadj : desc_[l], pool, z2));
    bwdr_.push_back(plans_of(desc_[l], dn, r == 0 ? opadj : desc_[r], pool, z2));
  }
}

std::vector<const GemmPlan*> Net::plans() const {
  std::vector<const GemmPlan*> out;
  for (size_t k = 0; k < fwd_.size(); ++k)
    for (const PlanSet* ps : {&fwd_[k], &bwdl_[k], &bwdr_[k]})
      for (int i = 0; i < ps->n; ++i) out.push_back(&ps->p[i]);
  return out;
}

namespace {
constexpr int EXT = -1;  // operator input/output, seed, root output, environment accumulators: double

// One product (its dense plan or each charge sector): node operands (internal
// nodes float in mixed mode, conjugated u/w leaves read conjugated for
// complex data).
void nrun(const Net& net, const NetBufs& b, const PlanSet& ps, const double* A, int an, const double* B, int bn,
          double* C, int cn, double alpha, double beta, cudaStream_t s) {
  auto internal = [&](int n) { return n >= net.nleaf() && n != EXT; };
  auto conj = [&](int n) {
    return n >= 0 && n < net.nleaf() && (net.role(n) == ROLE_UB || net.role(n) == ROLE_WB);
  };
  for (int i = 0; i < ps.n; ++i) {
    GettCall g = ps.p[i].proto;
    g.A = A;
    g.B = B;
    g.C = C;
    g.alpha = alpha;
    g.beta = beta;
    g.a32 = b.f32 && internal(an);
    g.b32 = b.f32 && internal(bn);
    g.c32 = b.f32 && internal(cn);
    g.cplx = b.cplx;
    g.a_conj = b.cplx && conj(an);
    g.b_conj = b.cplx && conj(bn);
    contract(g, *b.ex, s);
  }
}

const double* value(const Net& net, const NetBufs& b, int node) {
  return node < net.nleaf() ? b.leaf[node] : b.val[node];
}
}  // namespace

void net_prepare(const Net& net, NetBufs& b, cudaStream_t s) {
  for (int node = net.nleaf(); node < net.root(); ++node) {
    if (!net.fixed(node)) continue;
    const int l = net.left(node), r = net.right(node);
    nrun(net, b, net.fwd(node), value(net, b, l), l, value(net, b, r), r, b.val[node], node, 1.0, 0.0, s);
  }
}

void net_forward(const Net& net, NetBufs& b, double* out, double alpha, double beta, cudaStream_t s) {
  for (int node = net.nleaf(); node < net.root(); ++node) {
    if (net.fixed(node)) continue;
    const int l = net.left(node), r = net.right(node);
    nrun(net, b, net.fwd(node), value(net, b, l), l, value(net, b, r), r, b.val[node], node, 1.0, 0.0, s);
  }
  if (out) {
    const int node = net.root(), l = net.left(node), r = net.right(node);
    nrun(net, b, net.fwd(node), value(net, b, l), l, value(net, b, r), r, out, EXT, alpha, beta, s);
  }
}

void net_backward(const Net& net, NetBufs& b, const double* rho, bool need_op, double* op_out, double alpha_op,
                  bool need_env, double* du, double* dw, double alpha_env, cudaStream_t s) {
  std::vector<bool> need(net.nnode(), false);
  need[0] = need_op;
  for (int i = 1; i < net.nleaf(); ++i)
    need[i] = need_env && (net.role(i) == ROLE_UB || net.role(i) == ROLE_WB);
  for (int node = net.nleaf(); node < net.nnode(); ++node) need[node] = need[net.left(node)] || need[net.right(node)];
  for (int node = net.root(); node >= net.nleaf(); --node) {
    if (!need[node]) continue;
    const int l = net.left(node), r = net.right(node);
    const double* dn = node == net.root() ? rho : b.adj[node];
    const int dn_id = node == net.root() ? EXT : node;
    for (int side = 0; side < 2; ++side) {
      const int c = side == 0 ? l : r;
      if (!need[c]) continue;
      double* out;
      double alpha = 1.0, beta = 0.0;
      if (c == 0) {
        out = op_out;
        alpha = alpha_op;
        beta = 1.0;
      } else if (c < net.nleaf()) {
        out = net.role(c) == ROLE_UB ? du : dw;
        alpha = alpha_env;
        beta = 1.0;
      } else {
        out = b.adj[c];
      }
      const int out_id = c >= net.nleaf() ? c : EXT;
      if (side == 0)
        nrun(net, b, net.bwd_left(node), dn, dn_id, value(net, b, r), r, out, out_id, alpha, beta, s);
      else
        nrun(net, b, net.bwd_right(node), value(net, b, l), l, dn, dn_id, out, out_id, alpha, beta, s);
    }
  }
}

}  // namespace mera
