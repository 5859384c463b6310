// Host check of the library's seeded initialisation (mera::seeded_gaussians,
// mera::random_isometry), built by tests/test_init_host.py and linked against
// libmera.so; needs no GPU.  Prints, for a fixed set of cases, the normals and
// the isometries in full precision ("gauss seed stream count: values",
// "iso seed stream n p cplx z2: values"); the test compares them with
// oracle/rng.py.
#include "tn.h"

#include <cstdio>
#include <vector>

namespace {
std::vector<int> charges(const std::vector<int64_t>& dims) {
  int64_t n = 1;
  for (int64_t e : dims) n *= e;
  std::vector<int> ch(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = i;
    for (size_t j = dims.size(); j-- > 0;) {
      ch[i] ^= mera::z2_charge(r % dims[j], dims[j]);
      r /= dims[j];
    }
  }
  return ch;
}
}  // namespace

int main() {
  for (uint64_t seed : {0ull, 12345ull, 0xFFFFFFFFFFFFFFFFull}) {
    std::vector<double> g(7);
    mera::seeded_gaussians(seed, 5, 7, g.data());
    std::printf("gauss %llu 5 7:", (unsigned long long)seed);
    for (double x : g) std::printf(" %.17g", x);
    std::printf("\n");
  }
  struct Case {
    uint64_t seed, stream;
    int64_t n, p;
    int cplx, z2;
  };
  const Case cases[] = {{1, 0, 16, 16, 0, 0}, {1, 1, 16, 4, 0, 0}, {9, 3, 24, 6, 1, 0}, {9, 4, 10, 10, 1, 0},
                        {5, 1, 8, 4, 0, 1},   {5, 2, 8, 4, 1, 1}};
  for (const Case& c : cases) {
    std::vector<double> out(c.n * c.p * (c.cplx ? 2 : 1));
    const std::vector<int> rq = charges({2, 2, 2}), cq = charges({4});
    mera::random_isometry(c.seed, c.stream, c.n, c.p, c.cplx != 0, c.z2 ? rq.data() : nullptr,
                          c.z2 ? cq.data() : nullptr, out.data());
    std::printf("iso %llu %llu %lld %lld %d %d:", (unsigned long long)c.seed, (unsigned long long)c.stream,
                (long long)c.n, (long long)c.p, c.cplx, c.z2);
    for (double x : out) std::printf(" %.17g", x);
    std::printf("\n");
  }
  return 0;
}
