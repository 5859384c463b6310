// Contraction-tree executor for the binary MERA superoperators.
#pragma once
#include "common.h"
#include <map>
#include <memory>
#include <string>

namespace mera {

// A dense tensor layout: leg labels with extents and element strides.
struct TDesc {
  std::vector<int> legs;
  std::vector<int64_t> ext;
  std::vector<int64_t> stride;
  int64_t size() const {
    int64_t s = 1;
    for (auto e : ext) s *= e;
    return s;
  }
  int find(int leg) const {
    for (size_t i = 0; i < legs.size(); ++i)
      if (legs[i] == leg) return (int)i;
    return -1;
  }
};

// Device-resident offset tables, deduplicated by content.
class TablePool {
 public:
  // dry: count the bytes tables would take, allocate nothing (footprint queries)
  explicit TablePool(bool dry = false) : dry_(dry) {}
  // uploads are issued on this stream (ordered with the owner's kernels)
  void set_stream(cudaStream_t s) { stream_ = s; }
  // plans made with this pool also carry the real view of complex operands
  // (complex problems in a mixed-precision mode)
  void set_real_view(bool v) { real_view_ = v; }
  bool real_view() const { return real_view_; }
  const int64_t* get(const std::vector<int64_t>& host);
  size_t bytes() const { return bytes_; }

 private:
  bool dry_ = false;
  bool real_view_ = false;
  cudaStream_t stream_ = nullptr;
  std::map<std::vector<int64_t>, DevBuf> tables_;
  size_t bytes_ = 0;
};

// One pairwise contraction C = A x B, all index bookkeeping precomputed.
struct GemmPlan {
  GettCall proto;  // tables/strides/sizes; data pointers filled at run time
  double flops() const { return 2.0 * proto.M * proto.N * proto.K; }
};

// Z2 grading of a leg of extent e: index i has charge 1 iff i >= ceil(e/2)
// (the first half of a leg's basis even); a tuple of indices has the sum of
// its legs' charges mod 2.
inline int z2_charge(int64_t i, int64_t e) { return i >= (e + 1) / 2 ? 1 : 0; }

// Offsets in t's storage of the index tuples of the leg group `legs`
// (odometer order, last leg fastest); q >= 0 keeps only the tuples of Z2
// charge q, q < 0 keeps all.
std::vector<int64_t> sector_offsets(const TDesc& t, const std::vector<int>& legs, int q);

// The index bookkeeping of one contraction on the host, before upload.
// Groups: M = legs of C from A, N = legs of C from B (in C's order), K = legs
// shared by A and B (in B's order, except that the stride-1 leg of the larger
// operand that sums its stride-1 leg moves innermost).  A group is addressed by a table of
// offsets, or (affine) by index * stride.  q < 0: the dense contraction
// (affine groups detected); q = 0 or 1: the Z2 charge sector q, in which every
// group keeps its tuples of charge q (always tables).  For Z2-symmetric A and
// B (every entry of total charge 1 zero), C = A B is the sum of the two
// sectors, each writing only C's entries whose M and N tuples have charge q;
// the sectors hold a quarter of the dense multiply-adds.
struct HostGroup {
  std::vector<int64_t> table;  // empty when affine
  int64_t stride = 0;
  int64_t count = 0;
};
struct HostPlan {
  int64_t M = 0, N = 0, K = 0;
  HostGroup am, ak, bk, bn, cm, cn;
  int a_rfast = 0, b_rfast = 0;
  int c_rows = 0, c_vec = 1, c_rows_t = 0, c_vec_t = 1;  // output layout hints of GettCall
};
HostPlan host_plan(const TDesc& A, const TDesc& B, const TDesc& C, int q = -1);
// The same plan addressed in reals, for interleaved complex data: every
// offset and stride doubled (the real part of element e at 2e; the imaginary
// part is reached by offsetting the base pointer by one real), and the output
// hints of that view.
HostPlan real_view(const HostPlan& h);
// Uploads h's tables; with pool.real_view() also those of real_view(h).
GemmPlan upload_plan(const HostPlan& h, TablePool& pool);

// A complex product C = op(A) op(B) (op: conjugation or not) as four real
// products of the real views: Re C = Re A Re B - Im A Im B and
// Im C = Re A Im B + Im A Re B, the imaginary part of a conjugated operand
// entering with the opposite sign.  Part i multiplies component ca of A by
// component cb of B into component cc of C with the given sign; `first` marks
// the first write of a component (it takes the caller's beta, the second
// accumulates with beta = 1).
struct ComplexPart {
  int ca, cb, cc;
  double sign;
  bool first;
};
std::array<ComplexPart, 4> complex_parts(bool a_conj, bool b_conj);
// host_plan + upload_plan
GemmPlan make_plan(const TDesc& A, const TDesc& B, const TDesc& C, TablePool& pool, int q = -1);

// Ascending network of one side (A_L or A_R) of one layer.  Node numbering:
// 0..10 leaves (0 = operator; 1,3 = conj u; 2,5 = u; 4,7,9 = conj w;
// 6,8,10 = w), 11..20 internal nodes N1..N10 (20 = root = the ascended
// operator with legs [a b c A B C]).
class SideNet {
 public:
  static constexpr int NLEAF = 11, NNODE = 21, ROOT = 20;
  // chunk: slice length of the middle coarse leg b in the chi^9 chain
  // (N4 -> N5 -> N7 forward, dN7 -> dN5 -> dN3, dN4 backward); 0 = no slicing.
  SideNet(char side, int64_t chi_f, int64_t chi_c, TablePool& pool, int64_t chunk = 0);

  // Size (elements) of each internal node value and of each adjoint.
  int64_t node_size(int i) const { return desc_[i].size(); }
  // Elements a buffer for node i must hold (the 7-leg N5 only one slice).
  int64_t alloc_size(int i) const { return (sliced_ && i == 15) ? n5c_.size() : desc_[i].size(); }
  // Every plan that evaluations execute.
  std::vector<const GemmPlan*> executed_plans() const;
  bool sliced() const { return sliced_; }
  int64_t chunk() const { return nb_; }
  int64_t coarse() const { return cc_; }
  int64_t b_stride_n4() const { return sb4_; }
  int64_t b_stride_n7() const { return sb7_; }
  const GemmPlan& f5c() const { return f5c_; }
  const GemmPlan& f7c() const { return f7c_; }
  const GemmPlan& b7c() const { return b7c_; }
  const GemmPlan& b5lc() const { return b5lc_; }
  const GemmPlan& b5rc() const { return b5rc_; }
  static int left(int i) { return kids_[i - NLEAF][0]; }
  static int right(int i) { return kids_[i - NLEAF][1]; }

  // Forward/backward plans.
  const GemmPlan& fwd(int node) const { return fwd_[node - NLEAF]; }
  const GemmPlan& bwd_left(int node) const { return bwdl_[node - NLEAF]; }
  const GemmPlan& bwd_right(int node) const { return bwdr_[node - NLEAF]; }
  double forward_flops() const;
  char side() const { return side_; }

  static const int kids_[10][2];

 private:
  char side_;
  TDesc desc_[NNODE];
  GemmPlan fwd_[10], bwdl_[10], bwdr_[10];
  bool sliced_ = false;
  int64_t nb_ = 0, cc_ = 0, sb4_ = 0, sb7_ = 0;
  TDesc n5c_;
  GemmPlan f5c_, f7c_, b7c_, b5lc_, b5rc_;
};

// How contractions run: FP64 kernel, or tensor cores (3xTF32 / split-BF16)
// with operands packed into the workspace.
struct Exec {
  int prec = MERA_PREC_FP64;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* err = nullptr;  // device flag set by an expired bounded wait
  uint64_t wait_ns = 1000000000ull;  // limit of each tensor-core pipeline wait
  // two slots for packed operands that stay the same over a loop of products
  // (the loop-invariant factor of the sliced chain): packed once, reused
  void* keep[2] = {nullptr, nullptr};
  size_t keep_bytes[2] = {0, 0};
};
// An operand of a tensor-core product that is the same as in the previous
// call of the same loop: side 1 = A, 2 = B; valid = the slot already holds
// its planes (skip packing).
struct Keep {
  int side = 0;
  int slot = 0;
  bool valid = false;
};
void contract(const GettCall& g, const Exec& ex, cudaStream_t s, const Keep* keep = nullptr);
// The same plan for nb members (nb <= tc::TcEpilogue::MAXB) with different
// data (gs[k] differ only in data pointers and maximum words; their tables
// are equal): the tensor-core modes pack every member's operands and run one
// product launch over all of them, each member's arithmetic being that of
// contract(gs[k]); FP64 and complex products run member by member.
void contract_batch(const GettCall* gs, int nb, const Exec& ex, cudaStream_t s);
// Workspace a product needs (nb members batched).
size_t tc_workspace_bytes(const GettCall& g, int prec, int nb = 1);
// Bytes of the packed planes of one operand (side 1 = A, 2 = B) of g.
size_t tc_keep_bytes(const GettCall& g, int prec, int side);
// Keep-slot sizes the sliced chain of a SideNet needs (slot 0: N3, slot 1: N6).
void keep_need(const class SideNet& net, int prec, size_t need[2]);

// Buffers bound to a SideNet for one evaluation.  Leaves, root output,
// operator adjoint and u/w adjoints are double; internal node values and
// adjoints are float when f32 is set (mixed precision).
struct SideBufs {
  const double* leaf[SideNet::NLEAF] = {};  // leaf values (operator, u, conj u, w, conj w)
  double* val[SideNet::NNODE] = {};          // internal node values (root = output)
  double* adj[SideNet::NNODE] = {};          // adjoints (root = seed)
  bool f32 = false;
  bool cplx = false;   // interleaved complex data; conjugated leaves 1,3,4,7,9 read conjugated
  const Exec* ex = nullptr;
  // scaled split-FP16: 2 * NNODE device words, max|val[i]| at amax[i] and
  // max|adj[i]| at amax[NNODE + i] for internal nodes, written by the
  // products that store those buffers (null: operands are reduced when packed)
  unsigned* amax = nullptr;
};

// Batched forms: the same network for nb members (one SideBufs each, equal
// plans), every product one contract_batch over the members with the
// workspace of ex; out, op_out, du, dw: one pointer per member.  A sliced
// chain runs one member only.
void side_prepare_n(const SideNet& net, SideBufs* const* bs, int nb, const Exec& ex, cudaStream_t s);
void side_forward_n(const SideNet& net, SideBufs* const* bs, int nb, const Exec& ex, double* const* out,
                    double alpha, double beta, cudaStream_t s);
void side_backward_n(const SideNet& net, SideBufs* const* bs, int nb, const Exec& ex, bool need_op,
                     double* const* op_out, double alpha_op, bool need_env, double* const* du, double* const* dw,
                     double alpha_env, cudaStream_t s);

// Subtrees that do not contain the operator leaf: N1, N4, N6, N9.
void side_prepare(const SideNet& net, SideBufs& b, cudaStream_t s);
// Operator-dependent forward pass N2, N3, N5, N7, N8 (kept for the reverse
// pass) and, if out != nullptr, the root: out = beta*out + alpha*A_side(op).
void side_forward(const SideNet& net, SideBufs& b, double* out, double alpha, double beta,
                  cudaStream_t s);
// Reverse pass from the root adjoint.  need_op: adjoint of the operator
// (descending map) into op_out (alpha_op, accumulated); need_env: adjoints of
// the conjugated u/w copies accumulated into du/dw with alpha_env.
void side_backward(const SideNet& net, SideBufs& b, bool need_op, double* op_out, double alpha_op,
                   bool need_env, double* du, double* dw, double alpha_env, cudaStream_t s);

}  // namespace mera
