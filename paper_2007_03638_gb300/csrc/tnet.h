// A tensor network given as data: leaves with named legs and roles, and a
// pairwise contraction tree.  With z2 set, every leg carries the Z2 grading of
// tn.h (first half of its basis even) and every pairwise product runs as its
// two charge sectors (a quarter of the dense work), which is exact when the
// leaves and the seed are Z2-symmetric.  Used for the ternary MERA's three
// ascending networks and for Z2-symmetric binary problems (the binary
// network's default executor, which slices its chi^9 chain, is in tn.h).  One
// forward pass evaluates the ascended operator; one reverse pass seeded with
// the density matrix gives the descended operator (the adjoint of the
// operator leaf) and the environments (adjoints of the conjugated u and w
// leaves), with every product a contraction plan of tn.h.
#pragma once
#include "tn.h"

#include <array>
#include <string>
#include <vector>

namespace mera {

enum LeafRole { ROLE_OP = 0, ROLE_U = 1, ROLE_UB = 2, ROLE_W = 3, ROLE_WB = 4 };

struct NetDef {
  std::vector<std::string> legs;         // leaf legs; leaf 0 is the operator
  std::vector<int> role;                 // LeafRole per leaf
  std::vector<std::array<int, 2>> kids;  // internal node nleaf + k: its two children (earlier nodes)
  std::string out;                       // legs of the ascended operator, in storage order
  std::string rho;                       // legs of the seed (density matrix), in storage order
  std::string op_adj;                    // legs of the descended operator, in storage order
};

// The ternary MERA's networks A_L, A_C, A_R (side 'L', 'C', 'R').
NetDef ternary_netdef(char side);
// The binary MERA's networks A_L, A_R (side 'L', 'R'), for the executor below
// (unsliced chains: the Z2 charge sectors of binary problems).
NetDef binary_netdef(char side);

// The plans of one pairwise product: the dense plan, or its nonempty Z2
// charge sectors.
struct PlanSet {
  GemmPlan p[2];
  int n = 0;
};

class Net {
 public:
  // Coarse legs (a b c A B C) have extent cc, all others cf.
  Net(const NetDef& d, int64_t cf, int64_t cc, TablePool& pool, bool z2 = false);
  int nleaf() const { return nleaf_; }
  int nnode() const { return nnode_; }
  int root() const { return nnode_ - 1; }
  int left(int node) const { return kids_[node - nleaf_][0]; }
  int right(int node) const { return kids_[node - nleaf_][1]; }
  int role(int leaf) const { return role_[leaf]; }
  // true: the node's value does not involve the operator leaf (computed once per point)
  bool fixed(int node) const { return fixed_[node]; }
  int64_t size(int node) const { return desc_[node].size(); }
  const PlanSet& fwd(int node) const { return fwd_[node - nleaf_]; }
  const PlanSet& bwd_left(int node) const { return bwdl_[node - nleaf_]; }
  const PlanSet& bwd_right(int node) const { return bwdr_[node - nleaf_]; }
  std::vector<const GemmPlan*> plans() const;

 private:
  int nleaf_ = 0, nnode_ = 0;
  std::vector<std::array<int, 2>> kids_;
  std::vector<int> role_;
  std::vector<bool> fixed_;
  std::vector<TDesc> desc_;
  std::vector<PlanSet> fwd_, bwdl_, bwdr_;
};

// Buffers of one network for one layer: leaves (double), internal node
// values and adjoints (float when f32), complex flag, arithmetic.
struct NetBufs {
  std::vector<const double*> leaf;
  std::vector<double*> val, adj;  // indexed by node id (leaf entries unused)
  bool f32 = false;
  bool cplx = false;
  const Exec* ex = nullptr;
};

// Values of the nodes that do not involve the operator (once per point).
void net_prepare(const Net& net, NetBufs& b, cudaStream_t s);
// Values of the nodes that involve the operator; out = beta out + alpha A(op) if out.
void net_forward(const Net& net, NetBufs& b, double* out, double alpha, double beta, cudaStream_t s);
// Reverse pass seeded with rho: op_out += alpha_op D(rho) (if need_op),
// du/dw += alpha_env * environments of the conjugated u/w leaves (if need_env).
// Needs the values of net_forward for the environments, only those of
// net_prepare for the descended operator.
void net_backward(const Net& net, NetBufs& b, const double* rho, bool need_op, double* op_out, double alpha_op,
                  bool need_env, double* du, double* dw, double alpha_env, cudaStream_t s);

}  // namespace mera
