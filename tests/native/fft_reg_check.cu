// Host-side check of the register FFT (csrc/fft_reg.cuh) against a direct DFT in long double.
// Built and run by tests/test_fft_reg_host.py; prints one line per length and exits non-zero
// on a mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "../../paper_1507_05156_gb300/csrc/fft_reg.cuh"

using hse::cpx;

template <int N, int DIR, typename T>
static double check(unsigned seed) {
  cpx<T> a[N];
  long double xr[N], xi[N];
  srand(seed);
  for (int i = 0; i < N; ++i) {
    xr[i] = (long double)rand() / RAND_MAX - 0.5L;
    xi[i] = (long double)rand() / RAND_MAX - 0.5L;
    a[i] = {(T)xr[i], (T)xi[i]};
    xr[i] = (long double)a[i].x;
    xi[i] = (long double)a[i].y;
  }
  hse::fft<N, DIR, T>(a);
  double err = 0.0, nrm = 0.0;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < N; ++k) {
    long double sr = 0, si = 0;
    for (int n = 0; n < N; ++n) {
      const long double ang = DIR * 2.0L * pi * (long double)((n * k) % N) / N;
      sr += xr[n] * cosl(ang) - xi[n] * sinl(ang);
      si += xr[n] * sinl(ang) + xi[n] * cosl(ang);
    }
    err += (double)((a[k].x - sr) * (a[k].x - sr) + (a[k].y - si) * (a[k].y - si));
    nrm += (double)(sr * sr + si * si);
  }
  return std::sqrt(err / nrm);
}

template <int N>
static int run_len() {
  const double ef = std::fmax(check<N, -1, float>(N), check<N, +1, float>(N + 7));
  const double ed = std::fmax(check<N, -1, double>(3 * N), check<N, +1, double>(5 * N));
  const bool ok = ef < 1e-6 && ed < 1e-14;
  std::printf("N=%d float_err=%.3e double_err=%.3e %s\n", N, ef, ed, ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}

int main() {
  int bad = 0;
  bad += run_len<2>() + run_len<3>() + run_len<4>() + run_len<5>() + run_len<6>() + run_len<8>();
  bad += run_len<9>() + run_len<10>() + run_len<12>() + run_len<15>() + run_len<16>() + run_len<18>();
  bad += run_len<20>() + run_len<24>() + run_len<25>() + run_len<27>() + run_len<30>() + run_len<32>();
  return bad ? 1 : 0;
}
