// Seeded random isometries for mera_init_random: a counter-based generator
// (SplitMix64: Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) feeding Box-Muller normals, then the thin QR
// factor of the Gaussian matrix with R's diagonal made real and positive, the
// sign-fixed QR-of-Gaussian initialisation.  Host code: it runs once per
// problem, before any evaluation.
#include "common.h"

#include <cmath>
#include <complex>

namespace mera {
namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class T>
double abs2(const T& x) { return std::norm(x); }
template <>
double abs2<double>(const double& x) { return x * x; }

template <class T>
T conj_of(const T& x) { return std::conj(x); }
template <>
double conj_of<double>(const double& x) { return x; }

// x / |x| (1 for x = 0)
template <class T>
T phase(const T& x) {
  const double a = std::sqrt(abs2(x));
  return a > 0 ? x / a : T(1);
}

// Thin Q (n x p, row-major) of the row-major n x p matrix X (destroyed), with
// the diagonal of R real and positive: Householder reflectors H_k = 1 - 2 v v^dag
// on columns k = 0..p-1, Q = H_0 ... H_{p-1} [1_p; 0], then each column of Q
// times the phase of R_kk.
template <class T>
void thin_q(std::vector<T>& X, int64_t n, int64_t p, std::vector<T>& Q) {
  std::vector<std::vector<T>> vs(p);
  std::vector<T> rdiag(p);
  for (int64_t k = 0; k < p; ++k) {
    double nx = 0.0;
    for (int64_t i = k; i < n; ++i) nx += abs2(X[i * p + k]);
    nx = std::sqrt(nx);
    std::vector<T>& v = vs[k];
    v.assign(n - k, T(0));
    if (nx == 0.0) {
      rdiag[k] = T(0);
      continue;
    }
    const T alpha = -phase(X[k * p + k]) * nx;  // R_kk
    for (int64_t i = k; i < n; ++i) v[i - k] = X[i * p + k];
    v[0] -= alpha;
    double nv = 0.0;
    for (const T& x : v) nv += abs2(x);
    nv = std::sqrt(nv);
    if (nv == 0.0) {
      rdiag[k] = alpha;
      v.assign(n - k, T(0));
      continue;
    }
    for (T& x : v) x /= nv;
    for (int64_t j = k; j < p; ++j) {
      T s(0);
      for (int64_t i = k; i < n; ++i) s += conj_of(v[i - k]) * X[i * p + j];
      for (int64_t i = k; i < n; ++i) X[i * p + j] -= 2.0 * v[i - k] * s;
    }
    rdiag[k] = alpha;
  }
  Q.assign(n * p, T(0));
  for (int64_t k = 0; k < p; ++k) Q[k * p + k] = T(1);
  for (int64_t k = p; k-- > 0;) {
    const std::vector<T>& v = vs[k];
    for (int64_t j = 0; j < p; ++j) {
      T s(0);
      for (int64_t i = k; i < n; ++i) s += conj_of(v[i - k]) * Q[i * p + j];
      for (int64_t i = k; i < n; ++i) Q[i * p + j] -= 2.0 * v[i - k] * s;
    }
  }
  for (int64_t k = 0; k < p; ++k) {
    const T d = phase(rdiag[k]);
    for (int64_t i = 0; i < n; ++i) Q[i * p + k] *= d;
  }
}

// Element e of an interleaved array as T, and back.
template <class T>
T load(const double* a, int64_t e);
template <>
double load<double>(const double* a, int64_t e) { return a[e]; }
template <>
std::complex<double> load<std::complex<double>>(const double* a, int64_t e) { return {a[2 * e], a[2 * e + 1]}; }
void store(double* a, int64_t e, double v) { a[e] = v; }
void store(double* a, int64_t e, const std::complex<double>& v) {
  a[2 * e] = v.real();
  a[2 * e + 1] = v.imag();
}

// out = the sign-fixed thin Q of the n x p Gaussian matrix g, or, with
// charges, of each of its charge blocks (rows and columns of charge q, in
// ascending order), the entries between different charges zero.
template <class T>
void isometry_of(const double* g, int64_t n, int64_t p, const int* rq, const int* cq, double* out) {
  std::vector<T> X, Q;
  for (int q = 0; q < (rq ? 2 : 1); ++q) {
    std::vector<int64_t> rows, cols;
    for (int64_t i = 0; i < n; ++i)
      if (!rq || rq[i] == q) rows.push_back(i);
    for (int64_t j = 0; j < p; ++j)
      if (!cq || cq[j] == q) cols.push_back(j);
    if (cols.empty()) continue;
    if (rows.size() < cols.size())
      throw Error(MERA_ERR_ARG, "random isometry: a charge block with fewer rows than columns");
    const int64_t bn = (int64_t)rows.size(), bp = (int64_t)cols.size();
    X.assign(bn * bp, T(0));
    for (int64_t i = 0; i < bn; ++i)
      for (int64_t j = 0; j < bp; ++j) X[i * bp + j] = load<T>(g, rows[i] * p + cols[j]);
    thin_q(X, bn, bp, Q);
    for (int64_t i = 0; i < bn; ++i)
      for (int64_t j = 0; j < bp; ++j) store(out, rows[i] * p + cols[j], Q[i * bp + j]);
  }
}

}  // namespace

uint64_t splitmix64_output(uint64_t state, uint64_t k) { return mix64(state + k * GAMMA); }

void seeded_gaussians(uint64_t seed, uint64_t stream, int64_t count, double* out) {
  const uint64_t base = splitmix64_output(seed, stream + 1);
  for (int64_t j = 0; j < count; j += 2) {
    const double u1 = ((double)(splitmix64_output(base, (uint64_t)j + 1) >> 11) + 0.5) * 0x1p-53;
    const double u2 = ((double)(splitmix64_output(base, (uint64_t)j + 2) >> 11) + 0.5) * 0x1p-53;
    const double r = std::sqrt(-2.0 * std::log(u1)), t = 6.283185307179586 * u2;
    out[j] = r * std::cos(t);
    if (j + 1 < count) out[j + 1] = r * std::sin(t);
  }
}

void random_isometry(uint64_t seed, uint64_t stream, int64_t n, int64_t p, bool cplx, const int* row_charge,
                     const int* col_charge, double* out) {
  if (n < p || p < 1) throw Error(MERA_ERR_ARG, "random isometry: need rows >= columns >= 1");
  const int64_t count = n * p * (cplx ? 2 : 1);
  std::vector<double> g(count);
  seeded_gaussians(seed, stream, count, g.data());
  std::fill(out, out + count, 0.0);
  if (cplx)
    isometry_of<std::complex<double>>(g.data(), n, p, row_charge, col_charge, out);
  else
    isometry_of<double>(g.data(), n, p, row_charge, col_charge, out);
}

}  // namespace mera
