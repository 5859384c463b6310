// Internal declarations shared by the translation units of libmera.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <array>
#include <map>
#include <stdexcept>

#include "../../include/mera.h"

namespace mera {

// Error carrying a MERA_ERR_* code; thrown inside the library, converted to a
// return code at the C ABI.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& msg) : std::runtime_error(msg), code(c) {}
};

#define MERA_CUDA(call)                                                             \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess) {                                                        \
      throw ::mera::Error(_e == cudaErrorMemoryAllocation ? MERA_ERR_OOM : MERA_ERR_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(_e));      \
    }                                                                               \
  } while (0)

#define MERA_CHECK_LAUNCH() MERA_CUDA(cudaGetLastError())

// Per-object counters, reached through a thread-local pointer that the C ABI
// sets for the duration of each call.
struct Prof {
  int64_t launches = 0;
  int64_t gett_launches = 0;
  double gett_flops = 0.0;
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  size_t used = 0;              // events in use
  double gett_ms = 0.0;
  int64_t gett_timed = 0;
  int64_t energy_grad_calls = 0;
  // per-shape table of the timed contractions: key = (M, N, K, path)
  // with path = 0 FP64 GETT, else 1000 * (1 + kind) + 100 * store mode
  struct Shape {
    int64_t calls = 0;
    double ms = 0.0;
  };
  std::map<std::array<int64_t, 4>, Shape> shapes;
  std::vector<std::array<int64_t, 4>> pending;  // key of each recorded pair
  // Record an event pair around one contraction (if timing): call begin()
  // before the launch and end() after it.
  int64_t begin(int64_t M, int64_t N, int64_t K, cudaStream_t s);  // -1 when not timing
  void end(int64_t pair, int64_t path, cudaStream_t s);
  ~Prof();
  void collect();               // sum the recorded pairs (after a sync)
};
extern thread_local Prof* g_prof;
inline void count_launch(int n = 1) {
  if (g_prof) g_prof->launches += n;
}

// The device allocator every DevBuf uses (mera_set_allocator): null alloc
// means cudaMalloc / cudaFree.
struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*dealloc)(void*, void*) = nullptr;
  void* user = nullptr;
};
Allocator current_allocator();

// Owning device allocation; freed with the deallocator of the allocator that
// made it.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Allocator by;
  DevBuf() = default;
  explicit DevBuf(size_t n) { alloc(n); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), by(o.by) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; by = o.by; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t n) {
    release();
    if (n == 0) return;
    by = current_allocator();
    if (by.alloc) {
      p = by.alloc(n, by.user);
      if (!p) throw Error(MERA_ERR_OOM, "the device allocator returned no memory for " + std::to_string(n) + " bytes");
      if (reinterpret_cast<uintptr_t>(p) & 255) {
        by.dealloc(p, by.user);
        p = nullptr;
        throw Error(MERA_ERR_ARG, "the device allocator returned memory not aligned to 256 bytes");
      }
    } else {
      MERA_CUDA(cudaMalloc(&p, n));
    }
    bytes = n;
  }
  void release() {
    if (p) {
      if (by.alloc)
        by.dealloc(p, by.user);
      else
        cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------- GETT ----
// C[cm[m] + cn[n]] = alpha * sum_k A[am[m] + ak[k]] * B[bk[k] + bn[n]] + beta * C[..]
// Each index group is addressed through an int64 offset table, or, when the
// table pointer is null, through idx * stride.
struct GettOperand {
  const int64_t* t0 = nullptr;  // row-group table (M for A/C, K for B)
  const int64_t* t1 = nullptr;  // column-group table (K for A, N for B/C)
  int64_t s0 = 0, s1 = 0;       // strides used when a table is null
};
struct GettCall {
  const double* A = nullptr;
  GettOperand a;
  const double* B = nullptr;
  GettOperand b;
  double* C = nullptr;
  GettOperand c;
  int64_t M = 0, N = 0, K = 0;
  double alpha = 1.0, beta = 0.0;
  int a32 = 0, b32 = 0, c32 = 0;  // 1: operand stored as float (mixed-precision node buffers)
  int cplx = 0;                   // 1: interleaved complex elements (offsets count complex elements)
  int a_conj = 0, b_conj = 0;     // complex: use the complex conjugate of the operand
  int a_rfast = 0, b_rfast = 0;   // 1: the operand's stride-1 leg is in its row group (M for A, N for B)
  // Output layout hints for the tensor-core epilogue, fixed by the plan:
  // c_rows = 1: C's M-group offsets run contiguously through every aligned
  //   group of 32 rows (off(m) = off(m - m % 32) + m % 32);
  // c_vec = v (8, 4 or 1): N % v == 0, C's N-group offsets run contiguously
  //   through every aligned group of v columns, and every M-group offset and
  //   every group-start N offset is a multiple of v.
  int c_rows = 0, c_vec = 1;
  // the same hints for the transposed product C^T = B^T A^T (roles of the
  // M and N groups exchanged)
  int c_rows_t = 0, c_vec_t = 1;
  // Real view of complex operands, for the tensor-core path: the same groups
  // addressed in reals (the real part of element e at 2e, the imaginary part
  // at 2e + 1) and that view's output hints; has_rv = 0 when the plan has none.
  GettOperand ar, br, cr;
  int cr_rows = 0, cr_vec = 1, cr_rows_t = 0, cr_vec_t = 1;
  int has_rv = 0;
  // Largest magnitudes, as float bit patterns in device words (scaled
  // split-FP16 mode; ignored by the other modes): a_amax / b_amax, when set,
  // bound max|A| / max|B| (known from the operand's producer, so that the
  // packing need not reduce the operand first); c_amax, when set, receives
  // max|C| of the values this product stores (started at 0 when beta = 0,
  // unless c_amax_started: an earlier part of the same output already began it).
  const unsigned* a_amax = nullptr;
  const unsigned* b_amax = nullptr;
  unsigned* c_amax = nullptr;
  int c_amax_started = 0;
};
void gett_f64(const GettCall& g, cudaStream_t s);

// Plain row-major matrix product C = alpha op(A) op(B) + beta C with
// op = identity, transpose or conjugate transpose ('N'/'T'/'C'); leading
// dimensions are row strides in elements; cplx: interleaved complex data
// (alpha, beta real).
void gemm_f64(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha,
              const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
              double* C, int64_t ldc, cudaStream_t s, bool cplx = false);

// ---------------------------------------------------------- BLAS-1 etc ----
// Deterministic reductions: fixed grid, fixed per-thread ranges, two passes.
// Page-locked host memory (asynchronous device-to-host copies).
struct PinnedBuf {
  void* p = nullptr;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf&) = delete;
  PinnedBuf& operator=(const PinnedBuf&) = delete;
  ~PinnedBuf() { if (p) cudaFreeHost(p); }
  void alloc(size_t n) {
    if (p) cudaFreeHost(p);
    p = nullptr;
    MERA_CUDA(cudaMallocHost(&p, n));
  }
};

struct Reducer {
  DevBuf partial;    // per-block partial sums
  DevBuf result;     // device results
  std::vector<double> host;
  PinnedBuf pinned;  // results of the asynchronous forms
  int nblocks = 0;
  void init(int max_vectors);
  // Asynchronous forms of dots and trace (the same kernels and order): the
  // results reach pinned_results() when the stream gets there; the caller
  // synchronises the stream before reading them (several objects' reductions
  // then share one synchronisation).
  void dots_async(const double* X, int64_t ldx, int k, const double* y, int64_t n, cudaStream_t s);
  void trace_async(const double* a, int64_t n, cudaStream_t s);
  const double* pinned_results() const { return static_cast<const double*>(pinned.p); }
  // out[i] = sum_j X_i[j] * y[j] for i < k, where X_i = X + i*ldx
  void dots(const double* X, int64_t ldx, int k, const double* y, int64_t n, cudaStream_t s,
            double* out_host);
  double dot(const double* x, const double* y, int64_t n, cudaStream_t s);
  double trace(const double* a, int64_t n, cudaStream_t s);  // n x n matrix
  // complex: sum_j conj(x_j) y_j of n interleaved complex elements; trace of a complex matrix
  void dot_c(const double* x, const double* y, int64_t n, cudaStream_t s, double* re, double* im);
  void trace_c(const double* a, int64_t n, cudaStream_t s, double* re, double* im);
};
void axpy(double a, const double* x, double* y, int64_t n, cudaStream_t s);          // y += a x
void axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s); // y = a x + b y
void scal(double a, double* x, int64_t n, cudaStream_t s);
void fill(double v, double* x, int64_t n, cudaStream_t s);
void add_identity(double a, double* x, int64_t n, cudaStream_t s);   // x += a * 1 (n x n)
void symmetrize(double* x, int64_t n, cudaStream_t s);               // x = (x + x^T)/2
// y = sum_i c_i X_i   (c on device, length k), accumulate if beta==1
void combine(const double* X, int64_t ldx, int k, const double* c_dev, double* y, int64_t n,
             double beta, cudaStream_t s);
void copy(double* dst, const double* src, int64_t n, cudaStream_t s);
// partial traces of a 3-site operator (dim c per site, row-major)
void marginal_1site_mid(const double* r, int64_t c, double* out, cudaStream_t s);  // c x c
void marginal_2site_left(const double* r, int64_t c, double* out, cudaStream_t s); // c^2 x c^2
int check_finite(const double* x, int64_t n, cudaStream_t s);   // 1 if all finite
// ---- interleaved complex helpers (n = matrix order / element count) ----
void hermitize(double* x, int64_t n, cudaStream_t s);                      // x = (x + x^dag)/2
void add_identity_c(double re, double im, double* x, int64_t n, cudaStream_t s);
void marginal_1site_mid_c(const double* r, int64_t c, double* out, cudaStream_t s);
void marginal_2site_left_c(const double* r, int64_t c, double* out, cudaStream_t s);
// real symmetric embedding [[Re, -Im], [Im, Re]] of a complex n x n matrix (2n x 2n)
void embed_complex(const double* z, int64_t n, double* e, cudaStream_t s);
// complex n x n matrix from the left block column of a 2n x 2n embedding
void extract_complex(const double* e, int64_t n, double* z, cudaStream_t s);

// --------------------------------------------------------- small linalg ----
// Symmetric eigendecomposition of an n x n matrix (in place -> eigenvalues in
// evals_dev, eigenvectors as columns of V), cyclic parallel Jacobi in one CTA.
// Scratch of the eigensolver, kept by its owner so that no call allocates.
struct EigWork {
  DevBuf small, cs, red;
  DevBuf bar;           // grid-barrier words of the cooperative sweep (zeroed once)
  int coop_blocks = 0;  // resident blocks of the sweep kernel (0: not queried)
  std::map<int, DevBuf> sched;  // round-robin schedule per matrix size
};
void sym_eig(double* A, double* V, double* evals, int n, EigWork& w, cudaStream_t s);
// Same, optionally warm-started: with warm, V holds an orthogonal basis that
// A was already rotated into, and the result accumulates onto it.
void sym_eig_from(double* A, double* V, double* evals, int n, bool warm, EigWork& w, cudaStream_t s);

// ---------------------------------------------------------- seeded init ----
// k-th output (k >= 1) of SplitMix64 started at `state`.
uint64_t splitmix64_output(uint64_t state, uint64_t k);
// `count` standard normals of stream `stream` under `seed` (Box-Muller on
// pairs of uniforms from the SplitMix64 outputs; see mera_init_random).
void seeded_gaussians(uint64_t seed, uint64_t stream, int64_t count, double* out);
// out (n x p row-major, interleaved complex if cplx) = the sign-fixed thin QR
// factor of the seeded Gaussian matrix of stream `stream`; with row/column
// charges (Z2, may be null) the same per charge block, zero between charges.
void random_isometry(uint64_t seed, uint64_t stream, int64_t n, int64_t p, bool cplx, const int* row_charge,
                     const int* col_charge, double* out);

}  // namespace mera
