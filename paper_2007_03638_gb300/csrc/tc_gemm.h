// Tensor-core (tcgen05) contraction path: operand packing and the GEMM.
#pragma once
#include "common.h"
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace mera {
namespace tc {

// Operand planes: TF32 (hi/lo, kind::tf32), BF16 (hi/lo, kind::f16) or FP16
// (hi/lo of the operand scaled by a power of two, kind::f16).
enum { KIND_TF32 = 0, KIND_BF16 = 1, KIND_F16 = 2 };
inline int kind_elem(int kind) { return kind == KIND_TF32 ? 4 : 2; }
// Plane kind of a mixed-precision mode (mera_prec).
inline int kind_of_prec(int prec) {
  return prec == MERA_PREC_3XTF32 ? KIND_TF32 : prec == MERA_PREC_SPLIT_FP16 ? KIND_F16 : KIND_BF16;
}

// FP16 planes: the operand is multiplied by 2^e, e = 14 - E with
// max|x| = m 2^E (m in [0.5, 1)), so that its largest entry lies in
// [2^13, 2^14) and its low plane keeps 11 significant bits down to entries
// 2^-17 of the largest; amax_bits is the float bit pattern of max|x|.
// A zero or non-finite maximum gives e = 0; e is clamped to [-100, 100]
// (operands whose entries all lie below 2^-86 keep fewer bits).
__host__ __device__ inline int f16_scale_exp(unsigned amax_bits) {
  const unsigned ex = (amax_bits >> 23) & 0xFFu;
  if (ex == 0xFFu || (amax_bits & 0x7FFFFFFFu) == 0u) return 0;
  const int e = ex == 0u ? 100 : 14 - ((int)ex - 126);  // E = ex - 126 for m in [0.5, 1)
  return e > 100 ? 100 : (e < -100 ? -100 : e);
}

// Output side of one tensor-core contraction (offset tables as in GettCall).
struct TcEpilogue {
  int64_t M = 0, N = 0;
  int kblocks = 0;
  double alpha = 1.0, beta = 0.0;
  const int64_t* cm = nullptr;
  int64_t cms = 0;
  const int64_t* cn = nullptr;
  int64_t cns = 0;
  void* C = nullptr;
  int c_f64 = 0;       // 1: C is double, 0: float
  // layout hints (GettCall::c_rows / c_vec): rows = 1 when 32 consecutive
  // rows are 32 consecutive elements; vec = v when v consecutive columns
  // are v consecutive, v-aligned elements.  gemm_packed turns them into mode.
  int rows = 0, vec = 1;
  int mode = 0;        // store path: 0 staged transpose, 1 lanes = rows, 2/3 per-row 8/4-wide vectors
  // float C with beta != 0 in modes 1-3 and alpha a power of two: each lane
  // starts its register accumulator at (beta / alpha) C while the tile's MMAs
  // run, and the store writes alpha * acc without reading C again
  int preload = 0;
  float bscale = 0.f;  // beta / alpha (exact: alpha is a power of two)
  int* err = nullptr;  // set to 1 by a CTA whose bounded wait expired
  // FP16 planes: device words holding the float bits of max|A| and max|B|;
  // the products are divided by 2^(e_A + e_B) (f16_scale_exp) in the store
  const unsigned* a_amax = nullptr;
  const unsigned* b_amax = nullptr;
  // when set, every stored |C| value is folded into this word (atomicMax of
  // the float bits; split-K: by the reduction kernel)
  unsigned* c_amax = nullptr;
  uint64_t wait_ns = 1000000000ull;  // limit of each pipeline wait (default 1 s)
  // 8 bytes of device memory (zeroed by gemm_packed before the launch) from
  // which the CTAs take their work items in order; null: CTA c takes items
  // c, c + grid, ...  The items' arithmetic is the same either way.
  unsigned long long* work_ctr = nullptr;
  // split K (set by gemm_packed): ksplit slices of kbs K blocks, slice s
  // writing a plain row-major partial at C + s * split_stride
  int ksplit = 1, kbs = 0;
  int64_t split_stride = 0;
  // Batched products: nb members share the plan (shapes, tables, alpha,
  // beta) and differ in data.  Member b's A planes are rows
  // [b * a_member_rows, ...) of the A maps (B likewise), it writes
  // member_C[b] and its maxima are member_amax_a/b[b], member_cmax[b]
  // (gemm_packed fills member 0 from C, a_amax, b_amax, c_amax when nb = 1).
  static constexpr int MAXB = 8;
  int nb = 1;
  int64_t a_member_rows = 0, b_member_rows = 0;
  void* member_C[MAXB] = {};
  const unsigned* member_amax_a[MAXB] = {};
  const unsigned* member_amax_b[MAXB] = {};
  unsigned* member_cmax[MAXB] = {};
};

// Bytes of split-K partials gemm_packed may use for an M x N product.
size_t splitk_bytes(int64_t M, int64_t N, int64_t Kp, int kind);

// K rounded up to the 128-byte K block of the kind (32 TF32 / 64 BF16 values).
int64_t padded_k(int64_t K, int kind);

// Split src[r_off(r) + k_off(k)] (r < R, k < K; zero elsewhere) into hi/lo
// planes of [Rp x Kp] row-major tensor-core values.
// rows_fast: the source's stride-1 index runs along r (a tiled transpose keeps
// both the reads and the plane writes coalesced).  Kp must be a multiple of
// 32 and Rp of 64 (padded_k and round_up(., 128) give both).  KIND_F16: amax
// (a device word) receives the float bits of max|src| over the view first,
// and the planes hold the operand scaled by 2^f16_scale_exp(amax).
// amax_known: a device word already bounding max|src| (no reduction pass;
// the planes use it, and amax is not written).
void pack_split(const void* src, bool src_f64, const int64_t* rt, int64_t rs, const int64_t* kt,
                int64_t ks, int64_t R, int64_t K, int64_t Rp, int64_t Kp, int kind, void* hi,
                void* lo, bool rows_fast, cudaStream_t s, unsigned* amax = nullptr,
                const unsigned* amax_known = nullptr);

// C tile loop over packed planes: A [Mp x Kp], B [Np x Kp] (both K-major),
// Mp a multiple of 128 covering M, Np a multiple of 128 covering N.
// Products with too few output tiles to fill the GPU split K over several
// CTAs (partials in splitk_ws, summed in a fixed order by a second kernel).
// Returns the path taken: the epilogue store mode.
int gemm_packed(int kind, int64_t M, int64_t N, int64_t Kp, const void* a_hi, const void* a_lo,
                int64_t Mp, const void* b_hi, const void* b_lo, int64_t Np, const TcEpilogue& ep,
                cudaStream_t s, float* splitk_ws = nullptr, size_t splitk_ws_bytes = 0);

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace tc
}  // namespace mera
