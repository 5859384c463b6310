// Small dense FP64 linear algebra for the geometry: symmetric
// eigendecomposition by cyclic Jacobi with the parallel (round-robin)
// ordering, in one CTA up to order 64 and as one cooperative multi-CTA
// launch per sweep above.  Used for the preconditioner's density matrices
// (n = chi^2 for disentanglers, chi for isometries) and for the thin SVD of
// Grassmann tangents (eigen-decomposition of X^dag X, n = chi).
#include "common.h"
#include <algorithm>
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
// same block of A and on the rotations of pairs a and b, so a round is a
// fully parallel step after a small step that computes the rotations.  A
// whole sweep (all rounds) runs in one cooperative launch with a grid
// barrier between the steps.

// Rotation (Golub-Van Loan symmetric Schur 2x2) of pair (p, q); q >= n: none.
__device__ __forceinline__ double2 jac_rotation(const double* A, int n, int2 pq) {
  const int p = pq.x, q = pq.y;
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
  return make_double2(c, sn);
}

// Work item i of a round's apply step: i < h*h a 2x2 block of A, else one
// row entry pair of V.
__device__ __forceinline__ void jac_apply_item(double* A, double* V, int n, const int2* pairs, int h,
                                               const double2* cs, int64_t i) {
  const int64_t nblk = (int64_t)h * h;
  if (i < nblk) {
    const int a = (int)(i / h), b = (int)(i % h);
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
  } else if (i < nblk + (int64_t)n * h) {
    const int64_t t = i - nblk;
    const int r = (int)(t / h), b = (int)(t % h);
    const int pb = pairs[b].x, qb = pairs[b].y;
    if (qb >= n) return;
    const double cb = cs[b].x, sb = cs[b].y;
    const double vp = V[(int64_t)r * n + pb], vq = V[(int64_t)r * n + qb];
    V[(int64_t)r * n + pb] = cb * vp - sb * vq;
    V[(int64_t)r * n + qb] = sb * vp + cb * vq;
  }
}

__device__ __forceinline__ uint64_t jac_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of a cooperative launch (every block resident).  bar[0]
// counts arrivals, bar[1] is the generation, bar[2] the error flag.  The wait
// is bounded (2 s) and also ends when another block has given up; false then.
// gen (thread 0 only) is this block's copy of the generation.
__device__ bool jac_grid_barrier(unsigned* bar, unsigned& gen) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const uint64_t t0 = jac_timer();
      for (uint32_t it = 1; *(volatile unsigned*)&bar[1] == gen; ++it) {
        if (*(volatile unsigned*)&bar[2]) { ok = 0; break; }
        if ((it & 255u) == 0 && jac_timer() - t0 > 2000000000ull) {
          atomicExch(&bar[2], 1u);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ++gen;
  }
  __syncthreads();
  return ok != 0;
}

// One cyclic Jacobi sweep: all m-1 rounds of the round-robin schedule.
__global__ __launch_bounds__(1024) void jac_sweep_k(double* A, double* V, int n, const int2* sched, int h,
                                                    int rounds, double2* cs, unsigned* bar) {
  unsigned gen = 0;
  if (threadIdx.x == 0) gen = *(volatile unsigned*)&bar[1];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t work = (int64_t)h * h + (int64_t)n * h;
  for (int r = 0; r < rounds; ++r) {
    const int2* pairs = sched + (int64_t)r * h;
    for (int64_t k = tid; k < h; k += nthr) cs[k] = jac_rotation(A, n, pairs[k]);
    if (!jac_grid_barrier(bar, gen)) return;
    for (int64_t i = tid; i < work; i += nthr) jac_apply_item(A, V, n, pairs, h, cs, i);
    if (!jac_grid_barrier(bar, gen)) return;
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
  if (!w.bar.p) {
    w.bar.alloc(4 * sizeof(unsigned));
    MERA_CUDA(cudaMemsetAsync(w.bar.p, 0, 4 * sizeof(unsigned), s));
  }
  DevBuf& dpairs = w.sched.at(n);
  DevBuf& dcs = w.cs;
  DevBuf& dred = w.red;
  if (!warm) {
    eye_k<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(V, n);
    count_launch();
  }
  // one block per SM at most (the grid barrier's cost grows with the block count)
  const int64_t work = (int64_t)h * h + (int64_t)n * h;
  if (!w.coop_blocks) {
    int dev = 0, nsm = 0, occ = 0;
    MERA_CUDA(cudaGetDevice(&dev));
    MERA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    MERA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jac_sweep_k, 1024, 0));
    if (occ < 1) throw Error(MERA_ERR_UNSUPPORTED, "sym_eig: sweep kernel cannot be resident");
    w.coop_blocks = nsm;
  }
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(w.coop_blocks, (work + 1023) / 1024));
  double* pA = A;
  double* pV = V;
  int nn = n, hh = h, rounds = m - 1;
  int2* psched = dpairs.as<int2>();
  double2* pcs = dcs.as<double2>();
  unsigned* pbar = w.bar.as<unsigned>();
  void* args[] = {&pA, &pV, &nn, &psched, &hh, &rounds, &pcs, &pbar};
  double red[2] = {0, 0};
  unsigned flag[4] = {0, 0, 0, 0};
  double scale = 0.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    MERA_CUDA(cudaMemsetAsync(dred.p, 0, 2 * sizeof(double), s));
    jac_offdiag_k<<<152, 256, 0, s>>>(A, n, dred.as<double>());
    count_launch();
    MERA_CUDA(cudaMemcpyAsync(red, dred.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MERA_CUDA(cudaMemcpyAsync(flag, w.bar.p, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MERA_CUDA(cudaStreamSynchronize(s));
    if (flag[2]) {
      MERA_CUDA(cudaMemsetAsync(w.bar.p, 0, 4 * sizeof(unsigned), s));
      MERA_CUDA(cudaStreamSynchronize(s));
      throw Error(MERA_ERR_DEVICE_TIMEOUT, "sym_eig: a bounded grid barrier wait expired");
    }
    if (sweep == 0) scale = std::max(red[0], red[1]);
    if (red[0] <= 1e-15 * (scale > 0 ? scale : 1.0)) break;
    MERA_CUDA(cudaLaunchCooperativeKernel((const void*)jac_sweep_k, dim3(nb), dim3(1024), args, 0, s));
    count_launch();
    MERA_CHECK_LAUNCH();
  }
  MERA_CUDA(cudaMemcpyAsync(flag, w.bar.p, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  if (flag[2]) {
    MERA_CUDA(cudaMemsetAsync(w.bar.p, 0, 4 * sizeof(unsigned), s));
    MERA_CUDA(cudaStreamSynchronize(s));
    throw Error(MERA_ERR_DEVICE_TIMEOUT, "sym_eig: a bounded grid barrier wait expired");
  }
  diag_k<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, n, evals);
  count_launch();
  MERA_CHECK_LAUNCH();
  MERA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mera
