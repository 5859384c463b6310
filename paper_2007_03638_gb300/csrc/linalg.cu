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

namespace {
// ----------------------------------------------- multi-CTA Jacobi rounds ---
// One round applies n/2 disjoint rotations J: A <- J^T A J, V <- V J.  Every
// 2x2 block (pair a rows, pair b columns) of the result depends only on the
// same block of A and on the rotations of pairs a and b, so a round is one
// fully parallel kernel after a small kernel that computes the rotations.
__global__ void jac_rot_k(const double* __restrict__ A, int n, const int2* __restrict__ pairs, int h,
                          double2* __restrict__ cs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= h) return;
  const int p = pairs[k].x, q = pairs[k].y;
  double c = 1.0, sn = 0.0;
  if (q < n) {
    const double apq = A[(int64_t)p * n + q];
    if (fabs(apq) > 1e-300) {
      const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
      const double tau = (aqq - app) / (2.0 * apq);
      const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      c = 1.0 / sqrt(1.0 + t * t);
      sn = t * c;
    }
  }
  cs[k] = make_double2(c, sn);
}

__global__ void jac_apply_k(double* __restrict__ A, double* __restrict__ V, int n,
                            const int2* __restrict__ pairs, int h, const double2* __restrict__ cs) {
  const int64_t nblk = (int64_t)h * h;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < nblk) {
    const int a = (int)(tid / h), b = (int)(tid % h);
    const int pa = pairs[a].x, qa = pairs[a].y, pb = pairs[b].x, qb = pairs[b].y;
    const double ca = cs[a].x, sa = cs[a].y, cb = cs[b].x, sb = cs[b].y;
    const bool ra = qa < n, rb = qb < n;
    double x00 = A[(int64_t)pa * n + pb];
    double x01 = rb ? A[(int64_t)pa * n + qb] : 0.0;
    double x10 = ra ? A[(int64_t)qa * n + pb] : 0.0;
    double x11 = (ra && rb) ? A[(int64_t)qa * n + qb] : 0.0;
    // rows: J^T
    const double y00 = ca * x00 - sa * x10, y10 = sa * x00 + ca * x10;
    const double y01 = ca * x01 - sa * x11, y11 = sa * x01 + ca * x11;
    // columns: J
    A[(int64_t)pa * n + pb] = cb * y00 - sb * y01;
    if (rb) A[(int64_t)pa * n + qb] = sb * y00 + cb * y01;
    if (ra) A[(int64_t)qa * n + pb] = cb * y10 - sb * y11;
    if (ra && rb) A[(int64_t)qa * n + qb] = sb * y10 + cb * y11;
  } else if (tid < nblk + (int64_t)n * h) {
    const int64_t t = tid - nblk;
    const int i = (int)(t / h), b = (int)(t % h);
    const int pb = pairs[b].x, qb = pairs[b].y;
    if (qb >= n) return;
    const double cb = cs[b].x, sb = cs[b].y;
    const double vp = V[(int64_t)i * n + pb], vq = V[(int64_t)i * n + qb];
    V[(int64_t)i * n + pb] = cb * vp - sb * vq;
    V[(int64_t)i * n + qb] = sb * vp + cb * vq;
  }
}

__global__ void jac_offdiag_k(const double* __restrict__ A, int n, double* out) {
  double off = 0.0, dia = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs(A[i]);
    if (i / n == i % n) dia = fmax(dia, v); else off = fmax(off, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
    dia = fmax(dia, __shfl_xor_sync(0xffffffffu, dia, o));
  }
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(off));
    atomicMax(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)__double_as_longlong(dia));
  }
}

__global__ void diag_k(const double* __restrict__ A, int n, double* __restrict__ ev) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ev[i] = A[(int64_t)i * n + i];
}

__global__ void eye_k(double* V, int n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (int64_t)n * n) V[i] = (i / n == i % n) ? 1.0 : 0.0;
}
}  // namespace

namespace {
// round-robin schedule of all n-1 (even m) rounds: pairs[r*h + k]
std::vector<int2> schedule(int n) {
  const int m = (n + 1) & ~1, h = m / 2;
  std::vector<int> top(h), bot(h);
  for (int i = 0; i < h; ++i) { top[i] = 2 * i; bot[i] = 2 * i + 1; }
  std::vector<int2> out;
  for (int r = 0; r < m - 1; ++r) {
    for (int k = 0; k < h; ++k) out.push_back(make_int2(std::min(top[k], bot[k]), std::max(top[k], bot[k])));
    if (h > 1) {
      const int last_top = top[h - 1], first_bot = bot[0];
      for (int k = h - 1; k > 1; --k) top[k] = top[k - 1];
      top[1] = first_bot;
      for (int k = 0; k < h - 1; ++k) bot[k] = bot[k + 1];
      bot[h - 1] = last_top;
    }
  }
  return out;
}
}  // namespace

void sym_eig(double* A, double* V, double* evals, int n, EigWork& w, cudaStream_t s) {
  sym_eig_from(A, V, evals, n, false, w, s);
}

// Symmetric eigendecomposition by cyclic Jacobi.  If warm, V holds an
// orthogonal starting basis that A has already been rotated into (A is then
// nearly diagonal); on exit V holds the accumulated eigenvectors.
void sym_eig_from(double* A, double* V, double* evals, int n, bool warm, EigWork& w, cudaStream_t s) {
  if (n <= 0) return;
  if (n <= 64) {
    // small problems: one CTA does every sweep
    if (warm) throw Error(MERA_ERR_ARG, "sym_eig_from: warm start needs n > 64");
    const int m = (n + 1) & ~1;
    const size_t need = sizeof(double) * m + sizeof(int) * m;
    if (w.small.bytes < need) w.small.alloc(need);
    jacobi_kernel<<<1, JT, 0, s>>>(A, V, evals, n, 40, w.small.as<double>(),
                                   reinterpret_cast<int*>(w.small.as<char>() + sizeof(double) * m));
    count_launch();
    MERA_CHECK_LAUNCH();
    MERA_CUDA(cudaStreamSynchronize(s));
    return;
  }
  const int m = (n + 1) & ~1, h = m / 2;
  if (!w.sched.count(n)) {
    const std::vector<int2> sched = schedule(n);
    DevBuf b(sizeof(int2) * sched.size());
    MERA_CUDA(cudaMemcpyAsync(b.p, sched.data(), sizeof(int2) * sched.size(), cudaMemcpyHostToDevice, s));
    MERA_CUDA(cudaStreamSynchronize(s));
    w.sched.emplace(n, std::move(b));
  }
  if (w.cs.bytes < sizeof(double2) * h) w.cs.alloc(sizeof(double2) * h);
  if (w.red.bytes < 2 * sizeof(double)) w.red.alloc(2 * sizeof(double));
  DevBuf& dpairs = w.sched.at(n);
  DevBuf& dcs = w.cs;
  DevBuf& dred = w.red;
  if (!warm) {
    eye_k<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(V, n);
    count_launch();
  }
  const int64_t work = (int64_t)h * h + (int64_t)n * h;
  const unsigned nb = (unsigned)((work + 255) / 256);
  double red[2] = {0, 0};
  double scale = 0.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    MERA_CUDA(cudaMemsetAsync(dred.p, 0, 2 * sizeof(double), s));
    jac_offdiag_k<<<152, 256, 0, s>>>(A, n, dred.as<double>());
    count_launch();
    MERA_CUDA(cudaMemcpyAsync(red, dred.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MERA_CUDA(cudaStreamSynchronize(s));
    if (sweep == 0) scale = std::max(red[0], red[1]);
    if (red[0] <= 1e-15 * (scale > 0 ? scale : 1.0)) break;
    for (int r = 0; r < m - 1; ++r) {
      const int2* pr = dpairs.as<int2>() + (int64_t)r * h;
      jac_rot_k<<<(unsigned)((h + 127) / 128), 128, 0, s>>>(A, n, pr, h, dcs.as<double2>());
      jac_apply_k<<<nb, 256, 0, s>>>(A, V, n, pr, h, dcs.as<double2>());
      count_launch(2);
    }
    MERA_CHECK_LAUNCH();
  }
  diag_k<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, n, evals);
  count_launch();
  MERA_CHECK_LAUNCH();
  MERA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mera
