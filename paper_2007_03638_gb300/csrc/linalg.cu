// Small dense FP64 linear algebra for the geometry: symmetric
// eigendecomposition by cyclic Jacobi with the parallel (round-robin)
// ordering, in one CTA.  Used for the preconditioner's density matrices
// (n = chi^2 for disentanglers, chi for isometries) and for the thin SVD of
// Grassmann tangents (eigen-decomposition of X^dag X, n = chi).
#include "common.h"
#include <cmath>

namespace mera {

namespace {
constexpr int JT = 1024;

__device__ double block_max(double v) {
  __shared__ double red[JT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) red[0] = r;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// A (n x n, symmetric, row-major) is diagonalised in place: on exit
// A = diag(evals) up to the convergence threshold and V holds the
// eigenvectors in its columns (A_in = V diag(evals) V^T).  m = n rounded up
// to even; index n (if n is odd) is a dummy that takes part in no rotation.
// pc/ps/pp/pq: per-pair scratch of m/2 entries.
__global__ __launch_bounds__(JT) void jacobi_kernel(double* A, double* V, double* evals, int n,
                                                    int max_sweeps, double* cs, int* pairs) {
  const int m = (n + 1) & ~1;
  const int h = m / 2;
  const int tid = threadIdx.x;
  for (int64_t i = tid; i < (int64_t)n * n; i += blockDim.x) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  // round-robin tournament: position 0 fixed, others rotate
  int* top = pairs;
  int* bot = pairs + h;
  for (int i = tid; i < h; i += blockDim.x) {
    top[i] = 2 * i;
    bot[i] = 2 * i + 1;
  }
  __syncthreads();
  double scale = 0.0;
  for (int64_t i = tid; i < (int64_t)n * n; i += blockDim.x) scale = fmax(scale, fabs(A[i]));
  scale = block_max(scale);
  const double tol = 1e-15 * (scale > 0 ? scale : 1.0);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int64_t i = tid; i < (int64_t)n * n; i += blockDim.x)
      if (i / n != i % n) off = fmax(off, fabs(A[i]));
    off = block_max(off);
    if (off <= tol) break;
    for (int round = 0; round < m - 1; ++round) {
      // rotation parameters (Golub-Van Loan symmetric Schur 2x2)
      for (int k = tid; k < h; k += blockDim.x) {
        int p = min(top[k], bot[k]), q = max(top[k], bot[k]);
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[(int64_t)p * n + q];
          if (fabs(apq) > 1e-300) {
            const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int64_t idx = tid; idx < (int64_t)h * n; idx += blockDim.x) {
        const int k = (int)(idx / n);
        const int j = (int)(idx % n);
        const int p = min(top[k], bot[k]), q = max(top[k], bot[k]);
        if (q >= n) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double ap = A[(int64_t)p * n + j], aq = A[(int64_t)q * n + j];
        A[(int64_t)p * n + j] = c * ap - s * aq;
        A[(int64_t)q * n + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int64_t idx = tid; idx < (int64_t)h * n; idx += blockDim.x) {
        const int k = (int)(idx / n);
        const int i = (int)(idx % n);
        const int p = min(top[k], bot[k]), q = max(top[k], bot[k]);
        if (q >= n) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        double ap = A[(int64_t)i * n + p], aq = A[(int64_t)i * n + q];
        A[(int64_t)i * n + p] = c * ap - s * aq;
        A[(int64_t)i * n + q] = s * ap + c * aq;
        ap = V[(int64_t)i * n + p];
        aq = V[(int64_t)i * n + q];
        V[(int64_t)i * n + p] = c * ap - s * aq;
        V[(int64_t)i * n + q] = s * ap + c * aq;
      }
      __syncthreads();
      // next pairing: rotate all positions except top[0]
      if (tid == 0 && h > 1) {
        const int last_top = top[h - 1];
        const int first_bot = bot[0];
        for (int k = h - 1; k > 1; --k) top[k] = top[k - 1];
        if (h > 1) top[1] = first_bot;
        for (int k = 0; k < h - 1; ++k) bot[k] = bot[k + 1];
        bot[h - 1] = last_top;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < n; i += blockDim.x) evals[i] = A[(int64_t)i * n + i];
}
}  // namespace

void sym_eig(double* A, double* V, double* evals, int n, cudaStream_t s) {
  if (n <= 0) return;
  const int m = (n + 1) & ~1;
  DevBuf scratch(sizeof(double) * m + sizeof(int) * m);
  int threads = JT;
  jacobi_kernel<<<1, threads, 0, s>>>(A, V, evals, n, 40, scratch.as<double>(),
                                      reinterpret_cast<int*>(scratch.as<char>() + sizeof(double) * m));
  count_launch();
  MERA_CHECK_LAUNCH();
  MERA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mera
