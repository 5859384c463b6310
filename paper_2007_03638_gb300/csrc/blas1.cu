// Vector kernels of the FP64 path: deterministic dot products / traces
// (fixed grid, fixed per-thread ranges, warp-shuffle block reduction, second
// pass in a fixed order), axpy-type updates, symmetrisation and the partial
// traces that give the per-tensor density matrices.
#include "common.h"
#include <mutex>

namespace mera {

namespace {
constexpr int RT = 256;        // threads per reduction block
constexpr int RBLOCKS = 608;   // 4 blocks per SM on 152 SMs

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double ws[RT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < RT / 32 ? ws[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// grid (nblk, k): partial[i*nblk + b] = sum over block b's range of X_i * y
__global__ void dots_partial(const double* __restrict__ X, int64_t ldx,
                             const double* __restrict__ y, int64_t n,
                             double* __restrict__ partial) {
  const int i = blockIdx.y;
  const double* x = X + (int64_t)i * ldx;
  double s = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * RT + threadIdx.x; j < n; j += (int64_t)gridDim.x * RT)
    s = fma(x[j], y[j], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = s;
}

__global__ void finish_partial(const double* __restrict__ partial, int nblk,
                               double* __restrict__ out) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += RT) s += partial[(int64_t)i * nblk + b];
  s = block_sum(s);
  if (threadIdx.x == 0) out[i] = s;
}

__global__ void trace_partial(const double* __restrict__ a, int64_t n, double* __restrict__ partial) {
  double s = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * RT + threadIdx.x; j < n; j += (int64_t)gridDim.x * RT)
    s += a[j * n + j];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void axpby_k(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

__global__ void scal_k(double a, double* x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

__global__ void fill_k(double v, double* x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void add_identity_k(double a, double* x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i * n + i] += a;
}

// x = (x + x^T)/2 through 32x32 tiles: block (bi, bj) with bi <= bj handles
// the tile pair (bi,bj) and (bj,bi).
__global__ void symmetrize_k(double* x, int64_t n) {
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  __shared__ double t1[32][33], t2[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    int64_t i = bi * 32 + r, j = bj * 32 + tx;
    t1[r][tx] = (i < n && j < n) ? x[i * n + j] : 0.0;
    int64_t i2 = bj * 32 + r, j2 = bi * 32 + tx;
    t2[r][tx] = (i2 < n && j2 < n) ? x[i2 * n + j2] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int64_t i = bi * 32 + r, j = bj * 32 + tx;
    const double v = 0.5 * (t1[r][tx] + t2[tx][r]);
    if (i < n && j < n) x[i * n + j] = v;
    int64_t i2 = bj * 32 + r, j2 = bi * 32 + tx;
    if (bi != bj && i2 < n && j2 < n) x[i2 * n + j2] = 0.5 * (t2[r][tx] + t1[tx][r]);
  }
}

// y = sum_i c_i X_i + beta * y
__global__ void combine_k(const double* __restrict__ X, int64_t ldx, int k,
                          const double* __restrict__ c, double* __restrict__ y, int64_t n,
                          double beta) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double s = beta == 0.0 ? 0.0 : beta * y[j];
    for (int i = 0; i < k; ++i) s = fma(c[i], X[(int64_t)i * ldx + j], s);
    y[j] = s;
  }
}

// r: (c^3 x c^3) legs [a b d ; A B D]; out[b, B] = sum_{a,d} r[a b d; a B d]
__global__ void marg1_k(const double* __restrict__ r, int64_t c, double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c * c) return;
  const int64_t b = idx / c, B = idx % c;
  const int64_t n3 = c * c * c;
  double s = 0.0;
  for (int64_t a = 0; a < c; ++a)
    for (int64_t d = 0; d < c; ++d) s += r[(a * c * c + b * c + d) * n3 + (a * c * c + B * c + d)];
  out[idx] = s;
}

// out[(a b), (A B)] = sum_d r[a b d; A B d]
__global__ void marg2_k(const double* __restrict__ r, int64_t c, double* __restrict__ out) {
  const int64_t c2 = c * c;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c2 * c2) return;
  const int64_t ab = idx / c2, AB = idx % c2;
  const int64_t n3 = c2 * c;
  double s = 0.0;
  for (int64_t d = 0; d < c; ++d) s += r[(ab * c + d) * n3 + (AB * c + d)];
  out[idx] = s;
}

__global__ void finite_k(const double* __restrict__ x, int64_t n, int* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *flag = 0;
}


// conj(x) . y for interleaved complex arrays: partial[0*nb + b] real, [1*nb + b] imaginary
__global__ void cdot_partial(const double2* __restrict__ x, const double2* __restrict__ y, int64_t n,
                             double* __restrict__ partial) {
  double sr = 0.0, si = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * RT + threadIdx.x; j < n; j += (int64_t)gridDim.x * RT) {
    const double2 a = x[j], b = y[j];
    sr = fma(a.x, b.x, fma(a.y, b.y, sr));
    si = fma(a.x, b.y, fma(-a.y, b.x, si));
  }
  sr = block_sum(sr);
  si = block_sum(si);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sr;
    partial[gridDim.x + blockIdx.x] = si;
  }
}

__global__ void ctrace_partial(const double2* __restrict__ a, int64_t n, double* __restrict__ partial) {
  double sr = 0.0, si = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * RT + threadIdx.x; j < n; j += (int64_t)gridDim.x * RT) {
    sr += a[j * n + j].x;
    si += a[j * n + j].y;
  }
  sr = block_sum(sr);
  si = block_sum(si);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sr;
    partial[gridDim.x + blockIdx.x] = si;
  }
}

__global__ void hermitize_k(double2* x, int64_t n) {
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  __shared__ double2 t1[32][33], t2[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    int64_t i = bi * 32 + r, j = bj * 32 + tx;
    t1[r][tx] = (i < n && j < n) ? x[i * n + j] : make_double2(0.0, 0.0);
    int64_t i2 = bj * 32 + r, j2 = bi * 32 + tx;
    t2[r][tx] = (i2 < n && j2 < n) ? x[i2 * n + j2] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int64_t i = bi * 32 + r, j = bj * 32 + tx;
    // (x + x^dag)/2: element (i,j) averages x_ij with conj(x_ji)
    const double2 a = t1[r][tx], b = t2[tx][r];
    if (i < n && j < n) x[i * n + j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    int64_t i2 = bj * 32 + r, j2 = bi * 32 + tx;
    const double2 c = t2[r][tx], d = t1[tx][r];
    if (bi != bj && i2 < n && j2 < n) x[i2 * n + j2] = make_double2(0.5 * (c.x + d.x), 0.5 * (c.y - d.y));
  }
}

__global__ void add_identity_c_k(double re, double im, double2* x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i * n + i].x += re;
    x[i * n + i].y += im;
  }
}

__global__ void marg1c_k(const double2* __restrict__ r, int64_t c, double2* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c * c) return;
  const int64_t b = idx / c, B = idx % c;
  const int64_t n3 = c * c * c;
  double2 s = make_double2(0.0, 0.0);
  for (int64_t a = 0; a < c; ++a)
    for (int64_t d = 0; d < c; ++d) {
      const double2 v = r[(a * c * c + b * c + d) * n3 + (a * c * c + B * c + d)];
      s.x += v.x;
      s.y += v.y;
    }
  out[idx] = s;
}

__global__ void marg2c_k(const double2* __restrict__ r, int64_t c, double2* __restrict__ out) {
  const int64_t c2 = c * c;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= c2 * c2) return;
  const int64_t ab = idx / c2, AB = idx % c2;
  const int64_t n3 = c2 * c;
  double2 s = make_double2(0.0, 0.0);
  for (int64_t d = 0; d < c; ++d) {
    const double2 v = r[(ab * c + d) * n3 + (AB * c + d)];
    s.x += v.x;
    s.y += v.y;
  }
  out[idx] = s;
}

__global__ void embed_k(const double2* __restrict__ z, int64_t n, double* __restrict__ e) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  const double2 v = z[idx];
  const int64_t m = 2 * n;
  e[i * m + j] = v.x;
  e[i * m + n + j] = -v.y;
  e[(n + i) * m + j] = v.y;
  e[(n + i) * m + n + j] = v.x;
}

__global__ void extract_k(const double* __restrict__ e, int64_t n, double2* __restrict__ z) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  const int64_t m = 2 * n;
  z[idx] = make_double2(e[i * m + j], e[(n + i) * m + j]);
}

inline int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}
}  // namespace

void Reducer::init(int max_vectors) {
  nblocks = RBLOCKS;
  partial.alloc(sizeof(double) * (size_t)nblocks * max_vectors);
  result.alloc(sizeof(double) * (size_t)max_vectors);
  host.resize(max_vectors);
  pinned.alloc(sizeof(double) * (size_t)max_vectors);
}

void Reducer::dots_async(const double* X, int64_t ldx, int k, const double* y, int64_t n, cudaStream_t s) {
  if ((size_t)k > host.size()) throw Error(MERA_ERR_ARG, "Reducer: too many vectors");
  int nb = (int)std::min<int64_t>(nblocks, std::max<int64_t>(1, (n + RT - 1) / RT));
  dim3 grid(nb, k);
  dots_partial<<<grid, RT, 0, s>>>(X, ldx, y, n, partial.as<double>());
  finish_partial<<<k, RT, 0, s>>>(partial.as<double>(), nb, result.as<double>());
  count_launch(2);
  MERA_CHECK_LAUNCH();
  MERA_CUDA(cudaMemcpyAsync(pinned.p, result.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
}

void Reducer::trace_async(const double* a, int64_t n, cudaStream_t s) {
  int nb = (int)std::min<int64_t>(nblocks, std::max<int64_t>(1, (n + RT - 1) / RT));
  trace_partial<<<nb, RT, 0, s>>>(a, n, partial.as<double>());
  finish_partial<<<1, RT, 0, s>>>(partial.as<double>(), nb, result.as<double>());
  count_launch(2);
  MERA_CHECK_LAUNCH();
  MERA_CUDA(cudaMemcpyAsync(pinned.p, result.p, sizeof(double), cudaMemcpyDeviceToHost, s));
}

void Reducer::dots(const double* X, int64_t ldx, int k, const double* y, int64_t n,
                   cudaStream_t s, double* out_host) {
  if ((size_t)k > host.size()) throw Error(MERA_ERR_ARG, "Reducer: too many vectors");
  int nb = (int)std::min<int64_t>(nblocks, std::max<int64_t>(1, (n + RT - 1) / RT));
  dim3 grid(nb, k);
  dots_partial<<<grid, RT, 0, s>>>(X, ldx, y, n, partial.as<double>());
  finish_partial<<<k, RT, 0, s>>>(partial.as<double>(), nb, result.as<double>());
  count_launch(2);
  MERA_CHECK_LAUNCH();
  MERA_CUDA(cudaMemcpyAsync(out_host, result.p, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
}

double Reducer::dot(const double* x, const double* y, int64_t n, cudaStream_t s) {
  double r;
  dots(x, 0, 1, y, n, s, &r);
  return r;
}

double Reducer::trace(const double* a, int64_t n, cudaStream_t s) {
  int nb = (int)std::min<int64_t>(nblocks, std::max<int64_t>(1, (n + RT - 1) / RT));
  trace_partial<<<nb, RT, 0, s>>>(a, n, partial.as<double>());
  finish_partial<<<1, RT, 0, s>>>(partial.as<double>(), nb, result.as<double>());
  count_launch(2);
  MERA_CHECK_LAUNCH();
  double r;
  MERA_CUDA(cudaMemcpyAsync(&r, result.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  return r;
}

void axpy(double a, const double* x, double* y, int64_t n, cudaStream_t s) {
  axpby_k<<<grid_for(n), 256, 0, s>>>(a, x, 1.0, y, n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s) {
  axpby_k<<<grid_for(n), 256, 0, s>>>(a, x, b, y, n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void scal(double a, double* x, int64_t n, cudaStream_t s) {
  scal_k<<<grid_for(n), 256, 0, s>>>(a, x, n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void fill(double v, double* x, int64_t n, cudaStream_t s) {
  fill_k<<<grid_for(n), 256, 0, s>>>(v, x, n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void add_identity(double a, double* x, int64_t n, cudaStream_t s) {
  add_identity_k<<<grid_for(n), 256, 0, s>>>(a, x, n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void symmetrize(double* x, int64_t n, cudaStream_t s) {
  const unsigned nt = (unsigned)((n + 31) / 32);
  symmetrize_k<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(x, n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void combine(const double* X, int64_t ldx, int k, const double* c_dev, double* y, int64_t n,
             double beta, cudaStream_t s) {
  combine_k<<<grid_for(n), 256, 0, s>>>(X, ldx, k, c_dev, y, n, beta);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void copy(double* dst, const double* src, int64_t n, cudaStream_t s) {
  MERA_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
}
void marginal_1site_mid(const double* r, int64_t c, double* out, cudaStream_t s) {
  marg1_k<<<(unsigned)((c * c + 255) / 256), 256, 0, s>>>(r, c, out);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void marginal_2site_left(const double* r, int64_t c, double* out, cudaStream_t s) {
  marg2_k<<<(unsigned)((c * c * c * c + 255) / 256), 256, 0, s>>>(r, c, out);
  count_launch();
  MERA_CHECK_LAUNCH();
}
int check_finite(const double* x, int64_t n, cudaStream_t s) {
  DevBuf f(sizeof(int));
  int one = 1;
  MERA_CUDA(cudaMemcpyAsync(f.p, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  finite_k<<<grid_for(n), 256, 0, s>>>(x, n, f.as<int>());
  count_launch();
  MERA_CHECK_LAUNCH();
  MERA_CUDA(cudaMemcpyAsync(&one, f.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  return one;
}


void Reducer::dot_c(const double* x, const double* y, int64_t n, cudaStream_t s, double* re, double* im) {
  int nb = (int)std::min<int64_t>(nblocks, std::max<int64_t>(1, (n + RT - 1) / RT));
  cdot_partial<<<nb, RT, 0, s>>>(reinterpret_cast<const double2*>(x), reinterpret_cast<const double2*>(y), n,
                                 partial.as<double>());
  finish_partial<<<2, RT, 0, s>>>(partial.as<double>(), nb, result.as<double>());
  count_launch(2);
  MERA_CHECK_LAUNCH();
  double r[2];
  MERA_CUDA(cudaMemcpyAsync(r, result.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  *re = r[0];
  *im = r[1];
}

void Reducer::trace_c(const double* a, int64_t n, cudaStream_t s, double* re, double* im) {
  int nb = (int)std::min<int64_t>(nblocks, std::max<int64_t>(1, (n + RT - 1) / RT));
  ctrace_partial<<<nb, RT, 0, s>>>(reinterpret_cast<const double2*>(a), n, partial.as<double>());
  finish_partial<<<2, RT, 0, s>>>(partial.as<double>(), nb, result.as<double>());
  count_launch(2);
  MERA_CHECK_LAUNCH();
  double r[2];
  MERA_CUDA(cudaMemcpyAsync(r, result.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MERA_CUDA(cudaStreamSynchronize(s));
  *re = r[0];
  *im = r[1];
}

void hermitize(double* x, int64_t n, cudaStream_t s) {
  const unsigned nt = (unsigned)((n + 31) / 32);
  hermitize_k<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(reinterpret_cast<double2*>(x), n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void add_identity_c(double re, double im, double* x, int64_t n, cudaStream_t s) {
  add_identity_c_k<<<grid_for(n), 256, 0, s>>>(re, im, reinterpret_cast<double2*>(x), n);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void marginal_1site_mid_c(const double* r, int64_t c, double* out, cudaStream_t s) {
  marg1c_k<<<(unsigned)((c * c + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(r), c,
                                                          reinterpret_cast<double2*>(out));
  count_launch();
  MERA_CHECK_LAUNCH();
}
void marginal_2site_left_c(const double* r, int64_t c, double* out, cudaStream_t s) {
  marg2c_k<<<(unsigned)((c * c * c * c + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(r), c,
                                                                   reinterpret_cast<double2*>(out));
  count_launch();
  MERA_CHECK_LAUNCH();
}
void embed_complex(const double* z, int64_t n, double* e, cudaStream_t s) {
  embed_k<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(z), n, e);
  count_launch();
  MERA_CHECK_LAUNCH();
}
void extract_complex(const double* e, int64_t n, double* z, cudaStream_t s) {
  extract_k<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(e, n, reinterpret_cast<double2*>(z));
  count_launch();
  MERA_CHECK_LAUNCH();
}
}  // namespace mera

// ------------------------------------------- allocation-free dot products --
// Some callers cannot allocate device memory at all (a host application that
// owns every byte of the GPU and hands out no allocator, code running where
// cudaMalloc's implicit device synchronisation is not allowed).  For them
// mera_dots_noalloc computes the same deterministic batched dot products as
// the library's reducer without a mera_t and without allocating: the
// per-block partial sums live in this file-scope device array, which every
// GPU that loads the library holds until the process exits.
namespace mera {
namespace {
constexpr int NOALLOC_MAX_K = 32;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_K * RBLOCKS + NOALLOC_MAX_K];
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
}  // namespace
}  // namespace mera

extern "C" int mera_dots_noalloc(const double* X, int64_t ldx, int k, const double* y, int64_t n,
                                 double* out, void* stream) {
  using namespace mera;
  if (!X || !y || !out || k < 1 || n < 0) return MERA_ERR_ARG;
  if (k > NOALLOC_MAX_K) return MERA_ERR_ARG;
  if (k > 1 && ldx < n) return MERA_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MERA_ERR_CUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MERA_ERR_UNSUPPORTED;
  void* base = nullptr;
  {
    // one-time set-up per device, with that device current: host code holds
    // only a stand-in for the array, so its device address is looked up
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MERA_ERR_CUDA;
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  double* partial = static_cast<double*>(base);
  double* result = partial + (int64_t)NOALLOC_MAX_K * RBLOCKS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (int)std::min<int64_t>(RBLOCKS, std::max<int64_t>(1, (n + RT - 1) / RT));
  // an error left pending by an earlier launch on this thread is reported
  // (and left in place) before anything is launched, so that the check after
  // the launches sees only this call's
  if (cudaPeekAtLastError() != cudaSuccess) return MERA_ERR_CUDA;
  // every partial slot read below is written by this call, so nothing needs clearing
  dots_partial<<<dim3(nb, k), RT, 0, s>>>(X, ldx, y, n, partial);
  finish_partial<<<k, RT, 0, s>>>(partial, nb, result);
  count_launch(2);
  if (cudaGetLastError() != cudaSuccess) return MERA_ERR_CUDA;
  if (cudaMemcpyAsync(out, result, sizeof(double) * k, cudaMemcpyDefault, s) != cudaSuccess)
    return MERA_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MERA_ERR_CUDA;
  return MERA_OK;
}

