// Tensor-core contraction kernel for the mixed-precision path (sm_103a).
//
// C[cm[m] + cn[n]] = alpha * sum_k A[m,k] B[k,n] + beta * C[..]
// with the operands split into two tensor-core-precision planes,
// x = hi + lo (hi = round(x), lo = round(x - hi)), and the product evaluated
// as hi*hi + hi*lo + lo*hi with FP32 accumulation:
//   3xTF32      kind::tf32, hi/lo TF32 (~22 significant bits per operand)
//   split-BF16  kind::f16 with BF16 planes (~16 significant bits)
//
// Data flow per CTA (one 128 x BN output tile):
//   * operands are packed beforehand (pack_split) into K-major planes
//     [rows x Kp] (Kp a multiple of the 128-byte K block), zero padded;
//   * warp 0 (one elected lane) streams K blocks of all four planes with TMA
//     (2-D tiled, 128-byte swizzle) into a STAGES-deep shared-memory ring,
//     completion tracked by mbarrier transaction counts;
//   * warp 1 (one elected lane) issues tcgen05.mma (M=128, N=BN) for the three
//     products into one FP32 accumulator in tensor memory and frees each ring
//     slot with tcgen05.commit;
//   * all four warps drain the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31 = tile rows) and scatter through the offset tables.
// Every mbarrier wait is bounded (about one second of %globaltimer); on
// expiry the CTA records an error code, stops issuing, waits (bounded) for
// its own copies and MMAs, frees its tensor memory and returns.
#include "common.h"
#include "tc_gemm.h"

#include <cmath>
#include <cstdlib>
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

namespace mera {
namespace tc {
namespace {

// compile-time tuning: bytes of K per pipeline stage row (128: 128-byte
// swizzle, 64 KB stages; 64: 64-byte swizzle, 32 KB stages), the stage
// count, and the 128-byte K blocks per folded accumulator group.  Measured
// at chi = 32: six 32 KB stages run the large products 20% and the split-K
// Gram products 50% slower than three 64 KB stages, so 128.
#ifndef MERA_TC_KB_BYTES
#define MERA_TC_KB_BYTES 128
#endif
#ifndef MERA_TC_STAGES
#define MERA_TC_STAGES (MERA_TC_KB_BYTES == 64 ? 6 : 3)
#endif
#ifndef MERA_TC_PROMOTE_TF32
#define MERA_TC_PROMOTE_TF32 1
#endif
#ifndef MERA_TC_PROMOTE_BF16
#define MERA_TC_PROMOTE_BF16 2
#endif
#ifndef MERA_TC_PROMOTE_F16
#define MERA_TC_PROMOTE_F16 2
#endif

constexpr int BM = 128;
constexpr int STAGES = MERA_TC_STAGES;
constexpr int KB_BYTES = MERA_TC_KB_BYTES;  // K block = one swizzle row of every operand tile row
static_assert(KB_BYTES == 64 || KB_BYTES == 128, "K block of 64 or 128 bytes");
// limit of the waits that drain this CTA's own copies and MMAs after an
// abort (they complete in microseconds; the limit only bounds a broken case)
constexpr uint64_t DRAIN_NS = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait of at most limit_ns nanoseconds; false on expiry.
// The timer is read once per 256 polls (try_wait itself suspends the warp
// for a while before it reports an incomplete phase); a limit below the
// time of 256 polls is checked at the first poll.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  const uint32_t every = limit_ns < 100000ull ? 0u : 255u;
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & every) == 0 && gtimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// mbar_wait that also gives up (false) as soon as *abort is set
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                                   const int* abort) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  const uint32_t every = limit_ns < 100000ull ? 0u : 255u;
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*(volatile const int*)abort) return false;
    if ((it & every) == 0 && gtimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile with KB_BYTES-byte swizzle,
// rows of KB_BYTES bytes, 8-row groups 8 * KB_BYTES bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)(16 >> 4) << 16;                   // leading byte offset (unused with swizzle)
  d |= (uint64_t)((8 * KB_BYTES) >> 4) << 32;       // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)(KB_BYTES == 128 ? 2 : 4) << 61;   // 128- or 64-byte swizzle
  return d;
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (KIND == KIND_TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// Instruction descriptor: FP32 accumulator, K-major A and B, M=128, N=BN.
// Operand format: TF32 = 2 (kind::tf32); BF16 = 1, F16 = 0 (kind::f16).
template <int KIND>
__host__ __device__ constexpr uint32_t operand_format() {
  return KIND == KIND_TF32 ? 2u : (KIND == KIND_BF16 ? 1u : 0u);
}
template <int KIND, int BN>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4)                                   // D format: F32
         | (operand_format<KIND>() << 7)             // A format
         | (operand_format<KIND>() << 10)            // B format
         | ((uint32_t)(BN >> 3) << 17)               // N / 8
         | ((uint32_t)(BM >> 4) << 24);              // M / 16
}

constexpr int NACC = 4;  // tensor-memory accumulator buffers (4 x 128 columns)
constexpr int IRING = 8; // work items published ahead by the producer

struct Smem {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t item_full[IRING];   // the producer published item[i]
  uint64_t item_empty[IRING];  // the MMA issuer and every epilogue warp have read it
  int64_t item[IRING];         // work item index, -1 = no more work
  uint64_t acc_full[NACC];
  uint64_t acc_empty[NACC];
  uint64_t drain;  // MMA completion after an abort
  uint32_t tmem;
  int abort;
};

// Persistent kernel, one CTA per SM.  Work items (member, K slice, output
// tile) are handed out in order by a device counter (ep.work_ctr; without
// one, CTA c takes items c, c + grid, ...): CTAs that read the same operand
// tiles get consecutive items and start them together, so the tiles they
// share are still in L2 when the last of them reads them, however unevenly
// the CTAs progressed on earlier items.  Every CTA loads its own operand tiles.  The producer
// warp takes the items and passes their indices to the MMA issuer and the
// epilogue warps through a small ring in shared memory.  Warp
// roles (320 threads): warp 0 TMA producer, warp 1 MMA issuer, warps 2..9 fold and store (warp w reads TMEM lanes
// 32*(w%4)..+31 = its rows, columns 64*((w-2)/4)..+63 of the accumulator).
// The shared-memory ring, the tensor-memory accumulator ring and their
// barriers run on across tiles, so loads and MMAs of tile i+1 proceed while
// tile i is being stored.
// The tensor cores' FP32 accumulation truncates, so each group of PROMOTE K
// blocks is accumulated into a fresh tensor-memory buffer and folded into
// FP32 registers with round-to-nearest adds; NACC buffers let the MMAs run up
// to NACC-1 groups ahead of the folding.
constexpr int EPI_WARPS = 8;
constexpr int NTHREADS = 32 * (2 + EPI_WARPS);
constexpr int STG = 16;  // columns per staged store chunk

template <int KIND, int BN>
__global__ __launch_bounds__(NTHREADS, 1) void tc_gemm_kernel(const __grid_constant__ CUtensorMap a_hi,
                                                         const __grid_constant__ CUtensorMap a_lo,
                                                         const __grid_constant__ CUtensorMap b_hi,
                                                         const __grid_constant__ CUtensorMap b_lo,
                                                         TcEpilogue ep) {
  constexpr int A_BYTES = BM * KB_BYTES;   // one plane, one K block
  constexpr int B_BYTES = BN * KB_BYTES;
  constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int KSTEP_BYTES = 32;          // bytes of K per MMA (8 tf32 / 16 bf16)
  constexpr int KSTEPS = KB_BYTES / KSTEP_BYTES;
  constexpr uint32_t TMEM_COLS = NACC * BN;
  // K blocks accumulated in one tensor-memory buffer before it is folded:
  // 128 bytes of K for TF32 (the truncation error then stays near FP32
  // level), 256 for BF16 (its split error, ~1e-5, dominates the truncation
  // of 128 products) and FP16 (measured)
  constexpr int PROMOTE =
      (KIND == KIND_TF32 ? MERA_TC_PROMOTE_TF32 : (KIND == KIND_BF16 ? MERA_TC_PROMOTE_BF16 : MERA_TC_PROMOTE_F16)) *
      (128 / KB_BYTES);
  constexpr int HC = BN / 2;               // columns per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* staging = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES);
  Smem* S = reinterpret_cast<Smem*>(staging + EPI_WARPS * 32 * (STG + 1));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t sn = (ep.N + BN - 1) / BN, sm_ = (ep.M + BM - 1) / BM;
  const int64_t nt1 = sn * sm_;                // output tiles of one member
  const int64_t per_member = nt1 * ep.ksplit;  // work items (tile, K slice) of one member
  const int64_t ntiles = per_member * ep.nb;   // work items of all members, member slowest
  const int64_t cid = blockIdx.x, ncl = gridDim.x;
  // output tile tt (rows past M or columns past N load zeros and store
  // nothing).  The dimension with fewer tiles runs
  // fastest, so CTAs working at the same time share the tiles of the long
  // operand, which streams through L2 once.
  const bool mfast = sm_ < sn;
  auto tile_of = [&](int64_t tt, int64_t& m0, int64_t& n0) {
    const int64_t cm = mfast ? tt % sm_ : tt / sn, cn = mfast ? tt / sm_ : tt % sn;
    m0 = cm * (int64_t)BM;
    n0 = cn * (int64_t)BN;
  };
  // K blocks of work item t: [kb_lo, kb_hi)
  auto krange = [&](int64_t t, int& lo, int& hi) {
    const int sp = (int)((t % per_member) / nt1);
    lo = ep.ksplit > 1 ? sp * ep.kbs : 0;
    hi = ep.ksplit > 1 ? min(ep.kblocks, lo + ep.kbs) : ep.kblocks;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&S->full[s], 1);
      mbar_init(&S->empty[s], 1);  // the MMA issuer's commit
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(&S->acc_full[b], 1);
      mbar_init(&S->acc_empty[b], EPI_WARPS);  // one arrival per epilogue warp
    }
    for (int i = 0; i < IRING; ++i) {
      mbar_init(&S->item_full[i], 1);
      mbar_init(&S->item_empty[i], 1 + EPI_WARPS);
    }
    mbar_init(&S->drain, 1);
    S->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S->tmem;

  int64_t issued_loads = 0;
  if (warp == 0) {
    if (lane == 0) {
      for (const CUtensorMap* mp : {&a_hi, &a_lo, &b_hi, &b_lo})
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mp)) : "memory");
      int64_t kbg = 0, nit = 0;
      bool stop = false;
      int64_t t = ep.work_ctr ? (int64_t)atomicAdd(ep.work_ctr, 1ull) : cid;
      for (;;) {
        // publish item t (or the end of the work) to the MMA issuer and the epilogue
        const int sl = (int)(nit % IRING);
        if (nit >= IRING &&
            !mbar_wait_or_abort(&S->item_empty[sl], (uint32_t)((nit / IRING) - 1) & 1, ep.wait_ns, &S->abort)) {
          atomicExch(&S->abort, 1);
          break;
        }
        S->item[sl] = t < ntiles ? t : -1;
        mbar_arrive(&S->item_full[sl]);
        ++nit;
        if (t >= ntiles) break;
        // the next item, taken now so that the counter's latency hides behind this item's loads
        const int64_t tn = ep.work_ctr ? (int64_t)atomicAdd(ep.work_ctr, 1ull) : t + ncl;
        int64_t m0l, n0l;
        tile_of(t % nt1, m0l, n0l);
        const int64_t mb = t / per_member;  // member
        const int m0 = (int)(m0l + mb * ep.a_member_rows), n0 = (int)(n0l + mb * ep.b_member_rows);
        int klo, khi;
        krange(t, klo, khi);
        for (int kb = klo; kb < khi; ++kb, ++kbg) {
          const int s = (int)(kbg % STAGES);
          if (kbg >= STAGES && !mbar_wait(&S->empty[s], (uint32_t)((kbg / STAGES) - 1) & 1, ep.wait_ns)) {
            atomicExch(&S->abort, 1);
            stop = true;
            break;
          }
          if (*(volatile int*)&S->abort) { stop = true; break; }
          uint8_t* st = base + s * STAGE_BYTES;
          mbar_expect_tx(&S->full[s], STAGE_BYTES);
          const int kx = kb * (KB_BYTES / (KIND == KIND_TF32 ? 4 : 2));
          tma_load_2d(&a_hi, &S->full[s], st, kx, m0);
          tma_load_2d(&a_lo, &S->full[s], st + A_BYTES, kx, m0);
          tma_load_2d(&b_hi, &S->full[s], st + 2 * A_BYTES, kx, n0);
          tma_load_2d(&b_lo, &S->full[s], st + 2 * A_BYTES + B_BYTES, kx, n0);
          issued_loads = kbg + 1;
        }
        if (stop) break;
        t = tn;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t ID = idesc<KIND, BN>();
      int64_t kbg = 0, gg = 0, nit = 0;
      bool stop = false;
      while (!stop) {
        const int sl = (int)(nit % IRING);
        if (!mbar_wait_or_abort(&S->item_full[sl], (uint32_t)(nit / IRING) & 1, ep.wait_ns, &S->abort)) {
          atomicExch(&S->abort, 1);
          break;
        }
        const int64_t t = *(volatile int64_t*)&S->item[sl];
        mbar_arrive(&S->item_empty[sl]);
        ++nit;
        if (t < 0) break;
        int klo, khi;
        krange(t, klo, khi);
        for (int kb = klo; kb < khi; ++kb, ++kbg) {
          const int s = (int)(kbg % STAGES);
          const bool first = ((kb - klo) % PROMOTE) == 0;
          const bool last = ((kb - klo) % PROMOTE) == PROMOTE - 1 || kb == khi - 1;
          const int b = (int)(gg % NACC);
          if (!mbar_wait(&S->full[s], (uint32_t)(kbg / STAGES) & 1, ep.wait_ns)) {
            atomicExch(&S->abort, 1);
            stop = true;
            break;
          }
          if (first && gg >= NACC && !mbar_wait(&S->acc_empty[b], (uint32_t)((gg / NACC) - 1) & 1, ep.wait_ns)) {
            atomicExch(&S->abort, 1);
            stop = true;
            break;
          }
          if (*(volatile int*)&S->abort) { stop = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(base + s * STAGE_BYTES);
          const uint32_t ahi = st, alo = st + A_BYTES, bhi = st + 2 * A_BYTES, blo = st + 2 * A_BYTES + B_BYTES;
          const uint32_t dt = tmem + (uint32_t)(b * BN);
#pragma unroll
          for (int k = 0; k < KSTEPS; ++k) {
            const uint32_t off = k * KSTEP_BYTES;
            // small products first, the dominant one last
            mma<KIND>(dt, sdesc_sw(alo + off), sdesc_sw(bhi + off), ID, (first && k == 0) ? 0u : 1u);
            mma<KIND>(dt, sdesc_sw(ahi + off), sdesc_sw(blo + off), ID, 1u);
            mma<KIND>(dt, sdesc_sw(ahi + off), sdesc_sw(bhi + off), ID, 1u);
          }
          mma_commit(&S->empty[s]);
          if (last) {
            mma_commit(&S->acc_full[b]);
            ++gg;
          }
        }
      }
    }
  } else {
    // fold and store
    const int q = warp & 3;                    // TMEM lane quarter
    const int half = (warp - 2) >> 2;          // column half of the accumulator
    const int row = q * 32 + lane;
    float* stg = staging + (warp - 2) * 32 * (STG + 1);
    int64_t gg = 0;
    bool ok = true;
    // FP16 planes hold 2^(e_A + e_B) times the operands' product: the store
    // divides by that power of two (exact), the preload multiplies by it
    double alpha_eff = ep.alpha;
    float bscale = ep.bscale;
    float smax = 0.f;  // largest |value| this thread stores for the current member
    int64_t cur = -1;  // member of the previous work item
    // fold smax into the member's maximum word (one atomic per warp)
    auto flush_max = [&](int64_t mb) {
      if (mb < 0 || ep.ksplit > 1 || !ep.member_cmax[mb]) return;
      unsigned m = __float_as_uint(smax);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
      }
      if (lane == 0 && m) atomicMax(ep.member_cmax[mb], m);
      smax = 0.f;
    };
    int64_t nit = 0;
    while (ok) {
      const int sl = (int)(nit % IRING);
      if (!mbar_wait_or_abort(&S->item_full[sl], (uint32_t)(nit / IRING) & 1, ep.wait_ns, &S->abort)) {
        ok = false;
        break;
      }
      const int64_t t = *(volatile int64_t*)&S->item[sl];
      __syncwarp();
      if (lane == 0) mbar_arrive(&S->item_empty[sl]);
      ++nit;
      if (t < 0) break;
      const int64_t mb = t / per_member;
      if (mb != cur) {
        flush_max(cur);
        cur = mb;
        alpha_eff = ep.alpha;
        bscale = ep.bscale;
        if (ep.member_amax_a[mb]) {
          const int k = f16_scale_exp(*ep.member_amax_a[mb]) + f16_scale_exp(*ep.member_amax_b[mb]);
          alpha_eff = ldexp(ep.alpha, -k);
          bscale = (float)ldexp((double)ep.bscale, k);
        }
      }
      void* const Cm = ep.member_C[mb];
      int64_t m0, n0;
      tile_of(t % nt1, m0, n0);
      int klo, khi;
      krange(t, klo, khi);
      const int gpt = (khi - klo + PROMOTE - 1) / PROMOTE;  // accumulator groups of this item
      // this lane's output row offset, loaded while the MMAs run
      const int64_t mrow = m0 + row;
      const bool rvalid = mrow < ep.M;
      const int64_t my_off = rvalid ? (ep.cm ? ep.cm[mrow] : mrow * ep.cms) : 0;
      const int64_t nbase = n0 + half * HC;  // first column of this warp's half
      float acc[HC];
#pragma unroll
      for (int j = 0; j < HC; ++j) acc[j] = 0.f;
      if (ep.preload && rvalid) {
        // acc = (beta / alpha) C: loads issued now, their latency hidden by this tile's MMAs
        const float* C = static_cast<const float*>(Cm);
        if (ep.mode == 1) {
#pragma unroll
          for (int j = 0; j < HC; ++j) {
            const int64_t n = nbase + j;
            if (n < ep.N) acc[j] = bscale * C[my_off + (ep.cn ? ep.cn[n] : n * ep.cns)];
          }
        } else if (ep.mode == 2) {
#pragma unroll
          for (int c = 0; c < HC / 8; ++c) {
            const int64_t n = nbase + 8 * c;
            if (n >= ep.N) continue;
            const float* p = C + my_off + (ep.cn ? ep.cn[n] : n);
            float o[8];
            asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]),
                           "=f"(o[7])
                         : "l"(p));
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[8 * c + j] = bscale * o[j];
          }
        } else {
#pragma unroll
          for (int c = 0; c < HC / 4; ++c) {
            const int64_t n = nbase + 4 * c;
            if (n >= ep.N) continue;
            const float4 o = *reinterpret_cast<const float4*>(C + my_off + (ep.cn ? ep.cn[n] : n));
            acc[4 * c] = bscale * o.x;
            acc[4 * c + 1] = bscale * o.y;
            acc[4 * c + 2] = bscale * o.z;
            acc[4 * c + 3] = bscale * o.w;
          }
        }
      }
      for (int g = 0; g < gpt; ++g, ++gg) {
        const int b = (int)(gg % NACC);
        if (!mbar_wait(&S->acc_full[b], (uint32_t)(gg / NACC) & 1, ep.wait_ns)) { ok = false; break; }
        if (*(volatile int*)&S->abort) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int c0 = 0; c0 < HC; c0 += 64) {
          // two 32-column loads in flight, one wait
          uint32_t r[64];
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + half * HC + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
              : "r"(taddr));
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]),
                "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]),
                "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]),
                "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]),
                "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
              : "r"(taddr + 32u));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 64; ++j) acc[c0 + j] += __uint_as_float(r[j]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&S->acc_empty[b])) : "memory");
      }
      if (!ok) break;
      const bool f64out = ep.c_f64 != 0, acc_c = ep.beta != 0.0 && !ep.preload;
      void* Cbase =
          ep.ksplit > 1 ? static_cast<void*>(static_cast<float*>(Cm) + ((t % per_member) / nt1) * ep.split_stride)
                        : Cm;
      const double alpha = alpha_eff, beta = ep.beta;
      const float alpha_f = (float)alpha_eff, beta_f = (float)ep.beta;
      if (ep.mode == 1) {
        // lanes = 32 consecutive rows = 32 consecutive elements: one
        // coalesced 128-byte (float) store per column, no transpose
#pragma unroll
        for (int c0 = 0; c0 < HC; c0 += 16) {
          int64_t co[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t n = nbase + c0 + j;
            co[j] = n < ep.N ? (ep.cn ? ep.cn[n] : n * ep.cns) : -1;
          }
          if (rvalid) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (co[j] < 0) continue;
              const int64_t idx = my_off + co[j];
              if (f64out) {
                double* C = static_cast<double*>(Cbase);
                const double v = alpha * (double)acc[c0 + j];
                const double o = acc_c ? fma(beta, C[idx], v) : v;
                C[idx] = o;
                smax = fmaxf(smax, fabsf((float)o));
              } else {
                float* C = static_cast<float*>(Cbase);
                const float v = alpha_f * acc[c0 + j];
                const float o = acc_c ? fmaf(beta_f, C[idx], v) : v;
                C[idx] = o;
                smax = fmaxf(smax, fabsf(o));
              }
            }
          }
        }
      } else if (ep.mode == 2 || ep.mode == 3) {
        // float output, V consecutive aligned columns per vector: each lane
        // writes its own row in 32-byte (V = 8) or 16-byte (V = 4) pieces
        const int V = ep.mode == 2 ? 8 : 4;
        float* C = static_cast<float*>(Cbase);
        int64_t co[HC / 4];
#pragma unroll
        for (int c = 0; c < HC / 4; ++c) {
          const int64_t n = nbase + (int64_t)c * V;
          co[c] = (c * V < HC && n < ep.N) ? (ep.cn ? ep.cn[n] : n) : -1;
        }
        if (rvalid) {
          if (V == 8) {
#pragma unroll
            for (int c = 0; c < HC / 8; ++c) {
              if (co[c] < 0) continue;
              float* p = C + my_off + co[c];
              float v[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) v[j] = alpha_f * acc[8 * c + j];
              if (acc_c) {
                float o[8];
                asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]),
                               "=f"(o[7])
                             : "l"(p));
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = fmaf(beta_f, o[j], v[j]);
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) smax = fmaxf(smax, fabsf(v[j]));
              asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                           "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                           : "memory");
            }
          } else {
#pragma unroll
            for (int c = 0; c < HC / 4; ++c) {
              if (co[c] < 0) continue;
              float4* p = reinterpret_cast<float4*>(C + my_off + co[c]);
              float4 v = make_float4(alpha_f * acc[4 * c], alpha_f * acc[4 * c + 1], alpha_f * acc[4 * c + 2],
                                     alpha_f * acc[4 * c + 3]);
              if (acc_c) {
                const float4 o = *p;
                v.x = fmaf(beta_f, o.x, v.x);
                v.y = fmaf(beta_f, o.y, v.y);
                v.z = fmaf(beta_f, o.z, v.z);
                v.w = fmaf(beta_f, o.w, v.w);
              }
              smax = fmaxf(smax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
              *p = v;
            }
          }
        }
      } else {
        // any layout: 16-column chunks transposed through shared memory so
        // that lanes 0-15 and 16-31 write 16 consecutive columns of two rows
        const unsigned rowmask = __ballot_sync(0xffffffffu, rvalid);
        const int cl = lane & 15, rsel = lane >> 4;
#pragma unroll
        for (int c0 = 0; c0 < HC; c0 += STG) {
#pragma unroll
          for (int j = 0; j < STG; ++j) stg[lane * (STG + 1) + j] = acc[c0 + j];
          __syncwarp();
          const int64_t n = nbase + c0 + cl;
          const bool nvalid = n < ep.N;
          const int64_t coff = nvalid ? (ep.cn ? ep.cn[n] : n * ep.cns) : 0;
          // all shuffles and staged reads first, then the independent stores
          int64_t ro[16];
          float tv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int r = 2 * j + rsel;
            ro[j] = __shfl_sync(0xffffffffu, my_off, r);
            tv[j] = stg[r * (STG + 1) + cl];
          }
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int r = 2 * j + rsel;
            if (!nvalid || !((rowmask >> r) & 1u)) continue;
            const int64_t idx = ro[j] + coff;
            if (f64out) {
              const double v = alpha * (double)tv[j];
              double* C = static_cast<double*>(Cbase);
              const double o = acc_c ? fma(beta, C[idx], v) : v;
              C[idx] = o;
              smax = fmaxf(smax, fabsf((float)o));
            } else {
              // float output: FP32 arithmetic (the FP64 pipe is a few ops per clock per SM)
              float* C = static_cast<float*>(Cbase);
              const float v = alpha_f * tv[j];
              const float o = acc_c ? fmaf(beta_f, C[idx], v) : v;
              C[idx] = o;
              smax = fmaxf(smax, fabsf(o));
            }
          }
        }
      }
    }
    if (!ok) atomicExch(&S->abort, 1);
    flush_max(cur);
  }
  __syncthreads();
  if (*(volatile int*)&S->abort) {
    if (threadIdx.x == 0) atomicExch(ep.err, 1);
    // drain this CTA's copies still in flight (at most the last STAGES)
    if (warp == 0 && lane == 0) {
      const int64_t lo = issued_loads > STAGES ? issued_loads - STAGES : 0;
      for (int64_t kb = lo; kb < issued_loads; ++kb)
        mbar_wait(&S->full[kb % STAGES], (uint32_t)(kb / STAGES) & 1, DRAIN_NS);
    }
    // and the MMAs it issued: a commit tracks every earlier tcgen05 operation
    // of the issuing thread, so tensor memory is freed only after they finish
    if (warp == 1 && lane == 0) {
      mma_commit(&S->drain);
      mbar_wait(&S->drain, 0, DRAIN_NS);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// ----------------------------------------------------------------- packing -
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split 8 consecutive values of one plane row into hi/lo and write them as
// one 16-byte (BF16, FP16) or 32-byte (TF32) piece per plane; i = row * Kp + k,
// k a multiple of 8.  FP16: the values are multiplied by 2^e first (exact).
// The values arrive as floats (an FP64 source is rounded once, to 24 bits:
// the two planes keep at most 22 of them), so the split is FP32 arithmetic.
template <int KIND>
__device__ __forceinline__ void store_split8(const float (&v)[8], void* hi, void* lo, int64_t i, int e) {
  if (KIND == KIND_F16) {
    uint32_t h2[4], l2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __half hh[2], ll[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const float y = ldexpf(v[2 * j + t], e);
        hh[t] = __float2half_rn(y);
        ll[t] = __float2half_rn(y - __half2float(hh[t]));
      }
      h2[j] = (uint32_t)__half_as_ushort(hh[0]) | ((uint32_t)__half_as_ushort(hh[1]) << 16);
      l2[j] = (uint32_t)__half_as_ushort(ll[0]) | ((uint32_t)__half_as_ushort(ll[1]) << 16);
    }
    *reinterpret_cast<uint4*>(static_cast<__half*>(hi) + i) = make_uint4(h2[0], h2[1], h2[2], h2[3]);
    *reinterpret_cast<uint4*>(static_cast<__half*>(lo) + i) = make_uint4(l2[0], l2[1], l2[2], l2[3]);
  } else if (KIND == KIND_TF32) {
    float h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      h[j] = tf32_round(v[j]);
      l[j] = tf32_round(v[j] - h[j]);
    }
    float4* ph = reinterpret_cast<float4*>(static_cast<float*>(hi) + i);
    float4* pl = reinterpret_cast<float4*>(static_cast<float*>(lo) + i);
    ph[0] = make_float4(h[0], h[1], h[2], h[3]);
    ph[1] = make_float4(h[4], h[5], h[6], h[7]);
    pl[0] = make_float4(l[0], l[1], l[2], l[3]);
    pl[1] = make_float4(l[4], l[5], l[6], l[7]);
  } else {
    uint32_t h2[4], l2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat16 a = __float2bfloat16_rn(v[2 * j]), b = __float2bfloat16_rn(v[2 * j + 1]);
      const __nv_bfloat16 la = __float2bfloat16_rn(v[2 * j] - __bfloat162float(a));
      const __nv_bfloat16 lb = __float2bfloat16_rn(v[2 * j + 1] - __bfloat162float(b));
      h2[j] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
      l2[j] = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
    }
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(hi) + i) = make_uint4(h2[0], h2[1], h2[2], h2[3]);
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(lo) + i) = make_uint4(l2[0], l2[1], l2[2], l2[3]);
  }
}

// hi/lo planes [Rp x Kp] (row-major, K fastest) of src[r_off[r] + k_off[k]],
// zero outside R x K.  Block 32 x 8: threadIdx.y picks one of 8 rows,
// threadIdx.x 8 consecutive k (256 k per block row).  Reads run along k (the
// source's stride-1 direction); an affine unit-stride k group with aligned
// rows is read with vector loads.
template <typename Src, int KIND>
__global__ void pack_split_kernel(const Src* __restrict__ src, const int64_t* __restrict__ rt, int64_t rs,
                                  const int64_t* __restrict__ kt, int64_t ks, int64_t R, int64_t K,
                                  int64_t Rp, int64_t Kp, void* hi, void* lo, const unsigned* amax) {
  const int64_t r = (int64_t)blockIdx.x * 8 + threadIdx.y;
  const int64_t k0 = ((int64_t)blockIdx.y * 32 + threadIdx.x) * 8;
  if (r >= Rp || k0 >= Kp) return;
  const int e = KIND == KIND_F16 ? f16_scale_exp(*amax) : 0;
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.f;
  if (r < R) {
    const int64_t roff = rt ? rt[r] : r * rs;
    constexpr int VW = 16 / sizeof(Src);  // elements per 16-byte load
    if (!kt && ks == 1 && k0 + 8 <= K && (reinterpret_cast<uintptr_t>(src + roff + k0) & 15) == 0) {
      const Src* p = src + roff + k0;
#pragma unroll
      for (int j = 0; j < 8; j += VW) {
        if (sizeof(Src) == 4) {
          const float4 q = *reinterpret_cast<const float4*>(p + j);
          v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
        } else {
          const double2 q = *reinterpret_cast<const double2*>(p + j);
          v[j] = (float)q.x; v[j + 1] = (float)q.y;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t k = k0 + j;
        if (k < K) v[j] = (float)src[roff + (kt ? kt[k] : k * ks)];
      }
    }
  }
  store_split8<KIND>(v, hi, lo, r * Kp + k0, e);
}

// Same packing through a 64 x 64 shared-memory tile, for sources whose
// stride-1 direction is r: reads run along r, writes along k (16 k per
// thread and plane).  Block 256 threads.
template <typename Src, int KIND>
__global__ void pack_split_tiled_kernel(const Src* __restrict__ src, const int64_t* __restrict__ rt,
                                        int64_t rs, const int64_t* __restrict__ kt, int64_t ks, int64_t R,
                                        int64_t K, int64_t Rp, int64_t Kp, void* hi, void* lo,
                                        const unsigned* amax) {
  __shared__ float tile[64][65];  // [k][r], converted to float on load
  __shared__ int64_t roffs[64];
  const int t = threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.x * 64, r0 = (int64_t)blockIdx.y * 64;
  if (t < 64) {
    const int64_t r = r0 + t;
    roffs[t] = r < R ? (rt ? rt[r] : r * rs) : -1;
  }
  __syncthreads();
  {
    const int rl = t & 63;
    const int64_t roff = roffs[rl];
#pragma unroll 4
    for (int kl = t >> 6; kl < 64; kl += 4) {
      const int64_t k = k0 + kl;
      tile[kl][rl] = (roff >= 0 && k < K) ? (float)src[roff + (kt ? kt[k] : k * ks)] : 0.f;
    }
  }
  __syncthreads();
  const int rl = t >> 2, kc = (t & 3) * 16;
  const int64_t r = r0 + rl;
  if (r >= Rp) return;
  const int e = KIND == KIND_F16 ? f16_scale_exp(*amax) : 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t k = k0 + kc + 8 * h;
    if (k >= Kp) break;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = tile[kc + 8 * h + j][rl];
    store_split8<KIND>(v, hi, lo, r * Kp + k, e);
  }
}

// max |src| over the view r < R, k < K (offsets as in the packing), as float
// bits into *amax (which starts at 0): non-negative floats order like their
// bit patterns, so an unsigned atomicMax of the bits is a float maximum; a
// NaN entry (bits above every finite value) makes the maximum NaN.  Threads
// run along the source's stride-1 index (k, or r when rows_fast).
template <typename Src>
__global__ void amax_kernel(const Src* __restrict__ src, const int64_t* __restrict__ rt, int64_t rs,
                            const int64_t* __restrict__ kt, int64_t ks, int64_t R, int64_t K, int rows_fast,
                            unsigned* amax) {
  __shared__ unsigned wmax[8];
  unsigned m = 0u;
  const int64_t F = rows_fast ? R : K, S = rows_fast ? K : R;
  for (int64_t j = blockIdx.y; j < S; j += gridDim.y) {
    const int64_t so = rows_fast ? (kt ? kt[j] : j * ks) : (rt ? rt[j] : j * rs);
#pragma unroll 4
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F; i += (int64_t)gridDim.x * blockDim.x) {
      const int64_t fo = rows_fast ? (rt ? rt[i] : i * rs) : (kt ? kt[i] : i * ks);
      const unsigned b = __float_as_uint(fabsf((float)src[so + fo]));
      m = b > m ? b : m;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wmax[w] > m ? wmax[w] : m;
    if (m) atomicMax(amax, m);
  }
}

// Sum of the split-K partials in a fixed order, then the real epilogue;
// blockIdx.y = member (its partials at part + member * ksplit * M * N, the
// FP16 scales already divided out by the product kernel).
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int ksplit, int64_t M, int64_t N,
                                     TcEpilogue ep) {
  const int64_t total = M * N;
  const int mb = blockIdx.y;
  const float* pm = part + (int64_t)mb * ksplit * total;
  float smax = 0.f;
  const double alpha = ep.alpha;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int sp = 0; sp < ksplit; ++sp) acc += pm[(int64_t)sp * total + i];
    const int64_t m = i / N, n = i % N;
    const int64_t idx = (ep.cm ? ep.cm[m] : m * ep.cms) + (ep.cn ? ep.cn[n] : n * ep.cns);
    if (ep.c_f64) {
      double* C = static_cast<double*>(ep.member_C[mb]);
      const double v = alpha * (double)acc;
      const double o = ep.beta != 0.0 ? fma(ep.beta, C[idx], v) : v;
      C[idx] = o;
      smax = fmaxf(smax, fabsf((float)o));
    } else {
      float* C = static_cast<float*>(ep.member_C[mb]);
      const float v = (float)alpha * acc;
      const float o = ep.beta != 0.0 ? fmaf((float)ep.beta, C[idx], v) : v;
      C[idx] = o;
      smax = fmaxf(smax, fabsf(o));
    }
  }
  if (ep.member_cmax[mb]) {
    unsigned m = __float_as_uint(smax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned y = __shfl_xor_sync(0xffffffffu, m, o);
      m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(ep.member_cmax[mb], m);
  }
}

// ------------------------------------------------------------- host side ---
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encode() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) throw Error(MERA_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
}

CUtensorMap make_map(const void* ptr, int64_t rows, int64_t kp, int kind, int box_rows) {
  const int elem = kind_elem(kind);
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(kp * elem)};
  const cuuint32_t box[2] = {(cuuint32_t)(KB_BYTES / elem), (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((kp * elem) & 15))
    throw Error(MERA_ERR_ARG, "tensor map: base or row pitch not 16-byte aligned");
  const CUtensorMapDataType dt = kind == KIND_TF32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : kind == KIND_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult r = g_encode(&m, dt, 2,
                        const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        KB_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(MERA_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

template <int KIND, int BN>
size_t smem_bytes() {
  return 1024 + (size_t)STAGES * (2 * BM * KB_BYTES + 2 * BN * KB_BYTES) +
         sizeof(float) * EPI_WARPS * 32 * (STG + 1) + sizeof(Smem) + 64;
}

int num_sms() {
  static int cached[64] = {};
  static std::mutex mu;
  int dev = 0;
  MERA_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
  int n = 0;
  MERA_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

// Persistent launch: one CTA per SM, at most one per work item.
template <int KIND, int BN>
void launch(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
            const TcEpilogue& ep, int64_t items, cudaStream_t s) {
  auto kern = tc_gemm_kernel<KIND, BN>;
  static bool configured[64] = {};  // per device: shared-memory limit raised
  static std::mutex mu;
  int dev = 0;
  MERA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(MERA_ERR_UNSUPPORTED, "tensor-core GEMM: device ordinal out of range");
  const size_t sm = smem_bytes<KIND, BN>();
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!configured[dev]) {
      MERA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      configured[dev] = true;
    }
  }
  const unsigned grid = (unsigned)std::min<int64_t>(items, num_sms());
  kern<<<grid, NTHREADS, sm, s>>>(ah, al, bh, bl, ep);
}

}  // namespace

int64_t padded_k(int64_t K, int kind) {
  // whole K blocks, and a multiple of 32 elements (the packing's unit)
  const int64_t kb = std::max(KB_BYTES / (kind == KIND_TF32 ? 4 : 2), 32);
  return (K + kb - 1) / kb * kb;
}

namespace {
template <int KIND>
void launch_pack(const void* src, bool src_f64, const int64_t* rt, int64_t rs, const int64_t* kt, int64_t ks,
                 int64_t R, int64_t K, int64_t Rp, int64_t Kp, void* hi, void* lo, bool rows_fast,
                 const unsigned* amax, cudaStream_t s) {
  if (rows_fast) {
    if (Rp / 64 > 65535) throw Error(MERA_ERR_UNSUPPORTED, "pack_split: too many rows");
    const dim3 grid((unsigned)((Kp + 63) / 64), (unsigned)(Rp / 64));
    if (src_f64)
      pack_split_tiled_kernel<double, KIND><<<grid, 256, 0, s>>>((const double*)src, rt, rs, kt, ks, R, K, Rp, Kp,
                                                                 hi, lo, amax);
    else
      pack_split_tiled_kernel<float, KIND><<<grid, 256, 0, s>>>((const float*)src, rt, rs, kt, ks, R, K, Rp, Kp,
                                                                hi, lo, amax);
  } else {
    if ((Kp + 255) / 256 > 65535) throw Error(MERA_ERR_UNSUPPORTED, "pack_split: K too long");
    const dim3 grid((unsigned)(Rp / 8), (unsigned)((Kp + 255) / 256)), blk(32, 8);
    if (src_f64)
      pack_split_kernel<double, KIND><<<grid, blk, 0, s>>>((const double*)src, rt, rs, kt, ks, R, K, Rp, Kp, hi,
                                                           lo, amax);
    else
      pack_split_kernel<float, KIND><<<grid, blk, 0, s>>>((const float*)src, rt, rs, kt, ks, R, K, Rp, Kp, hi, lo,
                                                          amax);
  }
  count_launch();
  MERA_CHECK_LAUNCH();
}
}  // namespace

void pack_split(const void* src, bool src_f64, const int64_t* rt, int64_t rs, const int64_t* kt, int64_t ks,
                int64_t R, int64_t K, int64_t Rp, int64_t Kp, int kind, void* hi, void* lo, bool rows_fast,
                cudaStream_t s, unsigned* amax, const unsigned* amax_known) {
  if (Kp % 32 || Rp % 64) throw Error(MERA_ERR_ARG, "pack_split: Kp must be a multiple of 32, Rp of 64");
  if (kind == KIND_F16 && amax_known) {
    launch_pack<KIND_F16>(src, src_f64, rt, rs, kt, ks, R, K, Rp, Kp, hi, lo, rows_fast, amax_known, s);
  } else if (kind == KIND_F16) {
    if (!amax) throw Error(MERA_ERR_ARG, "pack_split: FP16 planes need a word for the operand's maximum");
    MERA_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned), s));
    if (R > 0 && K > 0) {
      const int64_t F = rows_fast ? R : K, S = rows_fast ? K : R;
      const dim3 grid((unsigned)std::min<int64_t>((F + 255) / 256, 16), (unsigned)std::min<int64_t>(S, 8192));
      if (src_f64)
        amax_kernel<double><<<grid, 256, 0, s>>>((const double*)src, rt, rs, kt, ks, R, K, rows_fast ? 1 : 0, amax);
      else
        amax_kernel<float><<<grid, 256, 0, s>>>((const float*)src, rt, rs, kt, ks, R, K, rows_fast ? 1 : 0, amax);
      count_launch();
      MERA_CHECK_LAUNCH();
    }
    launch_pack<KIND_F16>(src, src_f64, rt, rs, kt, ks, R, K, Rp, Kp, hi, lo, rows_fast, amax, s);
  } else if (kind == KIND_TF32) {
    launch_pack<KIND_TF32>(src, src_f64, rt, rs, kt, ks, R, K, Rp, Kp, hi, lo, rows_fast, nullptr, s);
  } else {
    launch_pack<KIND_BF16>(src, src_f64, rt, rs, kt, ks, R, K, Rp, Kp, hi, lo, rows_fast, nullptr, s);
  }
}

namespace {
// which products take their work items from the device counter (compile-time
// tuning): 2 every product, 1 split-K products only, 0 none.  Measured at
// chi = 32: the counter lifts the split-K Gram products from 198 to 243
// TFLOP/s and slows the short-K products with many tiles by 7%, so 1.
#ifndef MERA_TC_COUNTER
#define MERA_TC_COUNTER 1
#endif
#ifndef MERA_TC_SPLITK_MAX
#define MERA_TC_SPLITK_MAX 64
#endif
constexpr int SPLITK_MAX = MERA_TC_SPLITK_MAX;
// Number of K slices for an M x N x Kp product.  Only products whose output
// tiles cover less than half of the GPU split; each slice keeps >= 16 K
// blocks of 128 bytes.  Long K is cut into slices of about 128 (at most
// SPLITK_MAX), so that the CTAs sharing an operand tile (consecutive items)
// stay close in time; from there, the count whose work items fill the SMs'
// last wave best is taken (the smallest of equally good ones).
int choose_split(int64_t M, int64_t N, int64_t Kp, int kind) {
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + 127) / 128);
  // counted in 128-byte K blocks whatever the pipeline's K block
  const int64_t kblocks = Kp * (kind == KIND_TF32 ? 4 : 2) / 128;
  const int64_t nsm = 152;
  if (tiles * 2 > nsm || kblocks < 32) return 1;
  const int64_t lo = (nsm + tiles - 1) / tiles;  // at least one wave
  const int64_t hi = std::min<int64_t>((int64_t)SPLITK_MAX, kblocks / 16);
  if (hi <= 1) return 1;
  const int64_t from = std::min(std::max(lo, kblocks / 128), hi);
  int64_t best = from;
  double best_eff = 0.0;
  for (int64_t sp = from; sp <= hi; ++sp) {
    const int64_t items = tiles * sp, waves = (items + nsm - 1) / nsm;
    const double eff = (double)items / (double)(waves * nsm);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = sp;
    }
    if (eff > 0.97) break;
  }
  return (int)best;
}
}  // namespace

size_t splitk_bytes(int64_t M, int64_t N, int64_t Kp, int kind) {
  const int sp = choose_split(M, N, Kp, kind);
  return sp > 1 ? sizeof(float) * (size_t)sp * (size_t)M * (size_t)N : 0;
}

int gemm_packed(int kind, int64_t M, int64_t N, int64_t Kp, const void* a_hi, const void* a_lo, int64_t Mp,
                 const void* b_hi, const void* b_lo, int64_t Np, const TcEpilogue& ep_in, cudaStream_t s,
                 float* splitk_ws, size_t splitk_ws_bytes) {
  load_encode();
  const int elem = kind_elem(kind);
  const int bn = 128;
  TcEpilogue ep = ep_in;
  ep.M = M;
  ep.N = N;
  ep.kblocks = (int)(Kp / (KB_BYTES / elem));
  const int nb = ep.nb;
  if (nb < 1 || nb > TcEpilogue::MAXB) throw Error(MERA_ERR_ARG, "gemm_packed: member count out of range");
  if (nb == 1) {
    ep.member_C[0] = ep.C;
    ep.member_amax_a[0] = ep.a_amax;
    ep.member_amax_b[0] = ep.b_amax;
    ep.member_cmax[0] = ep.c_amax;
  }
  ep.a_member_rows = Mp;
  ep.b_member_rows = Np;
  const int64_t mt = (M + BM - 1) / BM, nt = (N + bn - 1) / bn;
  if (Mp < mt * BM || Np < nt * bn) throw Error(MERA_ERR_ARG, "gemm_packed: operand padding too small");
  // the split count depends on one member's shape only, so that a member's
  // arithmetic is the same alone and batched
  int sp = choose_split(M, N, Kp, kind);
  if (sp > 1 && (!splitk_ws || splitk_ws_bytes < sizeof(float) * (size_t)sp * M * N * nb)) sp = 1;
  TcEpilogue run = ep;
  if (sp > 1) {
    run.ksplit = sp;
    run.kbs = (ep.kblocks + sp - 1) / sp;
    run.ksplit = (ep.kblocks + run.kbs - 1) / run.kbs;  // no empty slice
    run.split_stride = M * N;
    for (int b = 0; b < nb; ++b) {
      run.member_C[b] = splitk_ws + (size_t)b * run.ksplit * M * N;
      run.member_cmax[b] = nullptr;
    }
    run.C = run.member_C[0];
    run.c_f64 = 0;
    run.cm = nullptr;
    run.cms = N;
    run.cn = nullptr;
    run.cns = 1;
    run.alpha = 1.0;
    run.beta = 0.0;
    run.rows = N == 1;
    run.vec = N % 8 == 0 ? 8 : N % 4 == 0 ? 4 : 1;
  }
  // store path: lanes = rows when rows are contiguous, else per-row vectors
  // when the columns are (pointer alignment permitting), else the transpose;
  // every member's output has the same alignment class (they have the same
  // layout), checked here because the path decides the rounding of beta != 0
  auto align_class = [](const void* p) {
    const uintptr_t c = reinterpret_cast<uintptr_t>(p);
    return c % 32 == 0 ? 2 : c % 16 == 0 ? 1 : 0;
  };
  const int acls = align_class(run.member_C[0]);
  for (int b = 1; b < nb; ++b)
    if (align_class(run.member_C[b]) != acls)
      throw Error(MERA_ERR_ARG, "gemm_packed: members' outputs differ in alignment");
  if (run.rows)
    run.mode = 1;
  else if (!run.c_f64 && run.vec == 8 && acls == 2)
    run.mode = 2;
  else if (!run.c_f64 && run.vec >= 4 && acls >= 1)
    run.mode = 3;
  else
    run.mode = 0;
  {
    int ex = 0;
    const bool pow2 = run.alpha != 0.0 && std::frexp(run.alpha, &ex) == 0.5;
    run.preload = run.mode >= 1 && !run.c_f64 && run.beta != 0.0 && pow2;
    run.bscale = run.preload ? (float)(run.beta / run.alpha) : 0.f;
  }
  if (kind == KIND_F16)
    for (int b = 0; b < nb; ++b)
      if (!run.member_amax_a[b] || !run.member_amax_b[b])
        throw Error(MERA_ERR_ARG, "gemm_packed: FP16 planes need their operands' maxima");
  const CUtensorMap ah = make_map(a_hi, nb * Mp, Kp, kind, BM), al = make_map(a_lo, nb * Mp, Kp, kind, BM);
  const CUtensorMap bh = make_map(b_hi, nb * Np, Kp, kind, bn), bl = make_map(b_lo, nb * Np, Kp, kind, bn);
  const int64_t items = nb * mt * nt * run.ksplit;
  if (MERA_TC_COUNTER == 0 || (MERA_TC_COUNTER == 1 && run.ksplit == 1)) run.work_ctr = nullptr;
  if (run.work_ctr) MERA_CUDA(cudaMemsetAsync(run.work_ctr, 0, sizeof(unsigned long long), s));
  if (kind == KIND_TF32)
    launch<KIND_TF32, 128>(ah, al, bh, bl, run, items, s);
  else if (kind == KIND_BF16)
    launch<KIND_BF16, 128>(ah, al, bh, bl, run, items, s);
  else
    launch<KIND_F16, 128>(ah, al, bh, bl, run, items, s);
  count_launch();
  MERA_CHECK_LAUNCH();
  if (sp > 1) {
    const int64_t total = M * N;
    const dim3 blocks((unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), (unsigned)nb);
    // the partials are already divided by the FP16 scales (their kernel ran with them)
    TcEpilogue red = ep;
    for (int b = 0; b < nb; ++b) red.member_amax_a[b] = red.member_amax_b[b] = nullptr;
    splitk_reduce_kernel<<<blocks, 256, 0, s>>>(splitk_ws, run.ksplit, M, N, red);
    count_launch();
    MERA_CHECK_LAUNCH();
  }
  return run.mode;
}

}  // namespace tc
}  // namespace mera
