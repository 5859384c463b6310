// FP64 tensor contraction kernel (GEMM-like tensor-tensor, "GETT").
//
// Every pairwise contraction of the MERA networks is a matrix product over
// three index groups (free legs of A, contracted legs, free legs of B).  The
// legs of a group need not be adjacent or ordered in memory: each group is
// addressed through an offset table, so input and output permutations are
// folded into the loads and stores and no permuted copy of any tensor is
// ever made.  GB300's FP64 units are the bound of this path (a few DFMA per
// clock per SM), so the kernel is a plain register-blocked tile: 64x64 C
// tile, 16-deep K slices staged in shared memory, 4x4 outputs per thread.
#include "common.h"

namespace mera {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ int64_t off(const int64_t* t, int64_t s, int64_t i) {
  return t ? t[i] : i * s;
}

__global__ __launch_bounds__(NT) void gett_f64_kernel(GettCall g) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ int64_t am[BM], bn[BN], cm[BM], cn[BN], ak[BK], bk[BK];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  if (tid < BM) {
    const int64_t m = m0 + tid;
    am[tid] = m < g.M ? off(g.a.t0, g.a.s0, m) : 0;
    cm[tid] = m < g.M ? off(g.c.t0, g.c.s0, m) : 0;
  } else if (tid < BM + BN) {
    const int j = tid - BM;
    const int64_t n = n0 + j;
    bn[j] = n < g.N ? off(g.b.t1, g.b.s1, n) : 0;
    cn[j] = n < g.N ? off(g.c.t1, g.c.s1, n) : 0;
  }
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
    __syncthreads();
    if (tid < BK) {
      const int64_t k = k0 + tid;
      ak[tid] = k < g.K ? off(g.a.t1, g.a.s1, k) : 0;
      bk[tid] = k < g.K ? off(g.b.t0, g.b.s0, k) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int i = tid; i < BM * BK; i += NT) {
      const int mm = i % BM, kk = i / BM;
      const bool ok = (m0 + mm < g.M) && (k0 + kk < g.K);
      As[kk][mm] = ok ? g.A[am[mm] + ak[kk]] : 0.0;
    }
#pragma unroll
    for (int i = tid; i < BN * BK; i += NT) {
      const int nn = i % BN, kk = i / BN;
      const bool ok = (n0 + nn < g.N) && (k0 + kk < g.K);
      Bs[kk][nn] = ok ? g.B[bk[kk] + bn[nn]] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int mm = ty + 16 * i;
    if (m0 + mm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = tx + 16 * j;
      if (n0 + nn >= g.N) continue;
      const int64_t idx = cm[mm] + cn[nn];
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v = fma(g.beta, g.C[idx], v);
      g.C[idx] = v;
    }
  }
}

// Complex variant: interleaved (re, im) elements, offsets in complex
// elements, optional conjugation of either operand.  32x32 C tile per CTA,
// 2x2 complex outputs per thread (4 real FMAs per complex multiply-add).
constexpr int CM = 32, CN = 32, CK = 16;
__global__ __launch_bounds__(NT) void gett_c128_kernel(GettCall g) {
  __shared__ double2 As[CK][CM + 1];
  __shared__ double2 Bs[CK][CN + 1];
  __shared__ int64_t am[CM], bn[CN], cm[CM], cn[CN], ak[CK], bk[CK];
  const double2* A = reinterpret_cast<const double2*>(g.A);
  const double2* B = reinterpret_cast<const double2*>(g.B);
  double2* C = reinterpret_cast<double2*>(g.C);
  const double sa = g.a_conj ? -1.0 : 1.0, sb = g.b_conj ? -1.0 : 1.0;
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.x * CM;
  const int64_t n0 = (int64_t)blockIdx.y * CN;
  if (tid < CM) {
    const int64_t m = m0 + tid;
    am[tid] = m < g.M ? off(g.a.t0, g.a.s0, m) : 0;
    cm[tid] = m < g.M ? off(g.c.t0, g.c.s0, m) : 0;
  } else if (tid < CM + CN) {
    const int j = tid - CM;
    const int64_t n = n0 + j;
    bn[j] = n < g.N ? off(g.b.t1, g.b.s1, n) : 0;
    cn[j] = n < g.N ? off(g.c.t1, g.c.s1, n) : 0;
  }
  const int tx = tid & 15, ty = tid >> 4;
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int64_t k0 = 0; k0 < g.K; k0 += CK) {
    __syncthreads();
    if (tid < CK) {
      const int64_t k = k0 + tid;
      ak[tid] = k < g.K ? off(g.a.t1, g.a.s1, k) : 0;
      bk[tid] = k < g.K ? off(g.b.t0, g.b.s0, k) : 0;
    }
    __syncthreads();
    for (int i = tid; i < CM * CK; i += NT) {
      const int mm = i % CM, kk = i / CM;
      const bool ok = (m0 + mm < g.M) && (k0 + kk < g.K);
      double2 v = ok ? A[am[mm] + ak[kk]] : make_double2(0.0, 0.0);
      v.y *= sa;
      As[kk][mm] = v;
    }
    for (int i = tid; i < CN * CK; i += NT) {
      const int nn = i % CN, kk = i / CN;
      const bool ok = (n0 + nn < g.N) && (k0 + kk < g.K);
      double2 v = ok ? B[bk[kk] + bn[nn]] : make_double2(0.0, 0.0);
      v.y *= sb;
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < CK; ++kk) {
      double2 a[2], b[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 2; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int mm = ty + 16 * i;
    if (m0 + mm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int nn = tx + 16 * j;
      if (n0 + nn >= g.N) continue;
      const int64_t idx = cm[mm] + cn[nn];
      double2 v = make_double2(g.alpha * acc[i][j].x, g.alpha * acc[i][j].y);
      if (g.beta != 0.0) {
        const double2 c = C[idx];
        v.x = fma(g.beta, c.x, v.x);
        v.y = fma(g.beta, c.y, v.y);
      }
      C[idx] = v;
    }
  }
}
}  // namespace

void gett_f64(const GettCall& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return;
  if (g.K <= 0) {
    throw Error(MERA_ERR_ARG, "gett_f64: empty contraction");
  }
  const int tm = g.cplx ? CM : BM, tn = g.cplx ? CN : BN;
  const int64_t gx = (g.M + tm - 1) / tm, gy = (g.N + tn - 1) / tn;
  if (gy > 65535) throw Error(MERA_ERR_UNSUPPORTED, "gett_f64: N too large for grid");
  dim3 grid((unsigned)gx, (unsigned)gy);
  Prof* pr = g_prof;
  const int64_t pair = pr ? pr->begin(g.M, g.N, g.K, s) : -1;
  if (g.cplx)
    gett_c128_kernel<<<grid, NT, 0, s>>>(g);
  else
    gett_f64_kernel<<<grid, NT, 0, s>>>(g);
  if (pr) pr->end(pair, 0, s);
  if (pr) {
    pr->launches++;
    pr->gett_launches++;
    pr->gett_flops += (g.cplx ? 8.0 : 2.0) * (double)g.M * (double)g.N * (double)g.K;
  }
  MERA_CHECK_LAUNCH();
}

Prof::~Prof() {
  for (auto e : ev) cudaEventDestroy(e);
}

int64_t Prof::begin(int64_t M, int64_t N, int64_t K, cudaStream_t s) {
  if (!timing) return -1;
  if (used + 2 > ev.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      MERA_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
    }
  }
  const int64_t i = (int64_t)used;
  used += 2;
  MERA_CUDA(cudaEventRecord(ev[i], s));
  pending.push_back({M, N, K, 0});
  return i;
}

void Prof::end(int64_t pair, int64_t path, cudaStream_t s) {
  if (pair < 0) return;
  MERA_CUDA(cudaEventRecord(ev[pair + 1], s));
  pending[pair / 2][3] = path;
}

void Prof::collect() {
  for (size_t i = 0; i + 1 < used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) {
      if (pending[i / 2][2] > 0) {  // contractions only (phases have K = 0)
        gett_ms += ms;
        gett_timed++;
      }
      Shape& sh = shapes[pending[i / 2]];
      sh.calls++;
      sh.ms += ms;
    }
  }
  used = 0;
  pending.clear();
}

void gemm_f64(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
              cudaStream_t s, bool cplx) {
  GettCall g;
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
  g.A = A; g.B = B; g.C = C;
  g.cplx = cplx;
  // A: op(A)[m,k];  'N': A[m*lda + k], 'T'/'C': A[k*lda + m] ('C' also conjugates)
  if (ta == 'N') { g.a.s0 = lda; g.a.s1 = 1; } else { g.a.s0 = 1; g.a.s1 = lda; }
  if (tb == 'N') { g.b.s0 = ldb; g.b.s1 = 1; } else { g.b.s0 = 1; g.b.s1 = ldb; }
  g.a_conj = cplx && ta == 'C';
  g.b_conj = cplx && tb == 'C';
  g.c.s0 = ldc; g.c.s1 = 1;
  gett_f64(g, s);
}

}  // namespace mera
