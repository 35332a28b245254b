#include <cstdio>
#include <random>
#include "krylov_host.h"
using cd = std::complex<double>;
int main() {
  const int m = 40, k = 23;
  mtf::HostArnoldi ha(m, 2);
  std::mt19937 rng(3);
  std::normal_distribution<double> N(0, 1);
  ha.start(1, 2.5);
  std::vector<cd> Hbar(size_t(k + 1) * k, 0.0);  // column-major, ld k+1
  for (int j = 0; j < k; ++j) {
    std::vector<double> h(2 * (j + 1));
    for (auto& v : h) v = N(rng);
    const double sub = std::abs(N(rng)) + 0.1;
    for (int q = 0; q <= j; ++q) Hbar[size_t(j) * (k + 1) + q] = cd(h[2 * q], h[2 * q + 1]);
    Hbar[size_t(j) * (k + 1) + j + 1] = sub;
    ha.add_column(1, j, h.data(), sub);
  }
  std::vector<cd> Q(size_t(k + 1) * k), R(size_t(k) * k);
  ha.qr(1, k, Q.data(), R.data(), k);
  double err = 0, nrm = 0, orth = 0;
  for (int p = 0; p < k; ++p)
    for (int q = 0; q <= k; ++q) {
      cd acc = 0;
      for (int t = 0; t < k; ++t) acc += Q[size_t(t) * (k + 1) + q] * R[size_t(p) * k + t];
      err += std::norm(acc - Hbar[size_t(p) * (k + 1) + q]);
      nrm += std::norm(Hbar[size_t(p) * (k + 1) + q]);
    }
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) {
      cd acc = 0;
      for (int q = 0; q <= k; ++q) acc += std::conj(Q[size_t(a) * (k + 1) + q]) * Q[size_t(b) * (k + 1) + q];
      orth += std::norm(acc - (a == b ? 1.0 : 0.0));
    }
  std::printf("||QR - H|| / ||H|| = %.3e   ||Q^H Q - I|| = %.3e\n", std::sqrt(err / nrm), std::sqrt(orth));
  return (std::sqrt(err / nrm) < 1e-12 && std::sqrt(orth) < 1e-12) ? 0 : 1;
}
