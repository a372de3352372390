// fft_reg.cuh - fully unrolled mixed-radix (2, 3, 4, 5) complex DFT of a pencil held in
// registers (prime-factor algorithm across coprime factors, Cooley-Tukey within prime powers).  Used by every 3-D transform of the Fock-like term (Sec. II C, Eq. "Fock":
// the pair density is transformed, multiplied by the kernel and transformed back).
//
// Convention: fft<N, -1> computes X[k] = sum_n x[n] exp(-2 pi i n k / N) (no scaling);
// fft<N, +1> the same with exp(+...).  Input and output are in natural order.
//
// All loops are compile-time (static_for), so every twiddle factor is a constant folded
// into the instruction stream and trivial twiddles (1, -1, +-i) cost nothing.
#pragma once

#include <type_traits>
#include <utility>

namespace hse {

template <typename T>
struct cpx {
  T x, y;
};

// ---------------------------------------------------------------------------
// compile-time trigonometry: cos/sin(2 pi j / n) from the Taylor series of sin and
// cos on an argument reduced exactly (integer arithmetic) to [0, pi/4].
// ---------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 16; ++k) {
    term *= -x * x / double((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}

__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 16; ++k) {
    term *= -x * x / double((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}

// returns cos (which = 0) or sin (which = 1) of 2 pi j / n
__host__ __device__ constexpr double trig2pi(int j, int n, int which) {
  j %= n;
  if (j < 0) j += n;
  const int q = (4 * j) / n;        // quarter turns
  const int rnum = 4 * j - q * n;   // remainder: angle = pi/2 * (q + rnum / n)
  double c = 0.0, s = 0.0;
  if (2 * rnum <= n) {
    const double r = (kPi / 2) * double(rnum) / double(n);
    c = taylor_cos(r);
    s = taylor_sin(r);
  } else {
    const double r = (kPi / 2) * double(n - rnum) / double(n);
    c = taylor_sin(r);
    s = taylor_cos(r);
  }
  double cc = c, ss = s;
  if (q == 1) { cc = -s; ss = c; }
  if (q == 2) { cc = -c; ss = -s; }
  if (q == 3) { cc = s; ss = -c; }
  return which == 0 ? cc : ss;
}

template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(static_cast<F&&>(f));
  }
}

template <typename T>
__host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
// (DIR * i) * a
template <int DIR, typename T>
__host__ __device__ __forceinline__ cpx<T> mul_i(cpx<T> a) {
  if constexpr (DIR > 0) return {-a.y, a.x};
  else return {a.y, -a.x};
}

// a * exp(DIR * 2 pi i J / N)
template <int N, int J, int DIR, typename T>
__host__ __device__ __forceinline__ cpx<T> twiddle(cpx<T> a) {
  constexpr int j = ((J % N) + N) % N;
  if constexpr (j == 0) {
    return a;
  } else if constexpr (2 * j == N) {
    return {-a.x, -a.y};
  } else if constexpr (4 * j == N) {
    return mul_i<DIR>(a);
  } else if constexpr (4 * j == 3 * N) {
    return mul_i<-DIR>(a);
  } else {
    constexpr T c = T(trig2pi(j, N, 0));
    constexpr T s = T(DIR * trig2pi(j, N, 1));
    return {a.x * c - a.y * s, a.x * s + a.y * c};
  }
}

// ---------------------------------------------------------------------------
// radix butterflies: y_s = sum_r x_r exp(DIR 2 pi i r s / R)
// ---------------------------------------------------------------------------
template <int R, int DIR, typename T>
struct Butterfly;

template <int DIR, typename T>
struct Butterfly<2, DIR, T> {
  static __host__ __device__ __forceinline__ void run(cpx<T>* a) {
    const cpx<T> t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};

template <int DIR, typename T>
struct Butterfly<3, DIR, T> {
  static __host__ __device__ __forceinline__ void run(cpx<T>* a) {
    constexpr T h = T(0.5);
    constexpr T s = T(DIR * 0.866025403784438646763723170752936183);  // DIR sin(2 pi / 3)
    const cpx<T> t1 = cadd(a[1], a[2]);
    const cpx<T> t2 = csub(a[1], a[2]);
    const cpx<T> m = {a[0].x - h * t1.x, a[0].y - h * t1.y};
    const cpx<T> r = {-s * t2.y, s * t2.x};  // i s t2
    a[0] = cadd(a[0], t1);
    a[1] = cadd(m, r);
    a[2] = csub(m, r);
  }
};

template <int DIR, typename T>
struct Butterfly<4, DIR, T> {
  static __host__ __device__ __forceinline__ void run(cpx<T>* a) {
    const cpx<T> a0 = cadd(a[0], a[2]);
    const cpx<T> a1 = csub(a[0], a[2]);
    const cpx<T> b0 = cadd(a[1], a[3]);
    const cpx<T> b1 = mul_i<DIR>(csub(a[1], a[3]));
    a[0] = cadd(a0, b0);
    a[2] = csub(a0, b0);
    a[1] = cadd(a1, b1);
    a[3] = csub(a1, b1);
  }
};

template <int DIR, typename T>
struct Butterfly<5, DIR, T> {
  static __host__ __device__ __forceinline__ void run(cpx<T>* a) {
    constexpr T c1 = T(trig2pi(1, 5, 0));
    constexpr T c2 = T(trig2pi(2, 5, 0));
    constexpr T s1 = T(DIR * trig2pi(1, 5, 1));
    constexpr T s2 = T(DIR * trig2pi(2, 5, 1));
    const cpx<T> t1 = cadd(a[1], a[4]);
    const cpx<T> t2 = cadd(a[2], a[3]);
    const cpx<T> t3 = csub(a[1], a[4]);
    const cpx<T> t4 = csub(a[2], a[3]);
    const cpx<T> p1 = {a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y};
    const cpx<T> p2 = {a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y};
    // i (s1 t3 + s2 t4) and i (s2 t3 - s1 t4)
    const cpx<T> q1 = {-(s1 * t3.y + s2 * t4.y), s1 * t3.x + s2 * t4.x};
    const cpx<T> q2 = {-(s2 * t3.y - s1 * t4.y), s2 * t3.x - s1 * t4.x};
    a[0] = {a[0].x + t1.x + t2.x, a[0].y + t1.y + t2.y};
    a[1] = cadd(p1, q1);
    a[4] = csub(p1, q1);
    a[2] = cadd(p2, q2);
    a[3] = csub(p2, q2);
  }
};

__host__ __device__ constexpr int pick_radix(int n) {
  return (n % 4 == 0) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : n;
}

__host__ __device__ constexpr bool radix_ok(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  return n == 1;
}

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// Coprime split N = N1 * N2 for the prime-factor algorithm: N1 = the power-of-two part, or
// the power-of-three part when N is odd; 0 when N is a prime power (no split exists).
__host__ __device__ constexpr int pfa_n1(int n) {
  int p2 = 1;
  while (n % (p2 * 2) == 0) p2 *= 2;
  if (p2 > 1 && p2 < n) return p2;
  int p3 = 1;
  while (n % (p3 * 3) == 0) p3 *= 3;
  if (p3 > 1 && p3 < n) return p3;
  return 0;
}

// k in [0, n1*n2) with k = k1 (mod n1) and k = k2 (mod n2)  (Chinese remainder theorem)
__host__ __device__ constexpr int crt_index(int k1, int k2, int n1, int n2) {
  int k = 0;
  while (k % n1 != k1 || k % n2 != k2) ++k;
  return k;
}

template <int N, int DIR, typename T>
__host__ __device__ __forceinline__ void fft(cpx<T>* a);

// Cooley-Tukey (decimation in time) for prime powers: N = R * M with twiddles.
template <int N, int DIR, typename T>
__host__ __device__ __forceinline__ void fft_ct(cpx<T>* a) {
  constexpr int R = pick_radix(N);
  if constexpr (R == N) {
    Butterfly<N, DIR, T>::run(a);
  } else {
    constexpr int M = N / R;
    cpx<T> sub[R][M];
    static_for<0, R>([&](auto rc) {
      static_for<0, M>([&](auto mc) {
        sub[decltype(rc)::value][decltype(mc)::value] = a[decltype(mc)::value * R + decltype(rc)::value];
      });
    });
    static_for<0, R>([&](auto rc) { fft<M, DIR, T>(sub[decltype(rc)::value]); });
    static_for<0, M>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      cpx<T> t[R];
      static_for<0, R>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        t[r] = twiddle<N, r * k, DIR, T>(sub[r][k]);
      });
      Butterfly<R, DIR, T>::run(t);
      static_for<0, R>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        a[k + M * s] = t[s];
      });
    });
  }
}

// Prime-factor (Good-Thomas) algorithm for N = N1 * N2 with gcd(N1, N2) = 1: input index
// n = (N2 n1 + N1 n2) mod N, output index k = CRT(k1, k2); the 2-D DFT of size N1 x N2 that
// remains needs no twiddle factors.
template <int N, int DIR, typename T>
__host__ __device__ __forceinline__ void fft_pfa(cpx<T>* a) {
  constexpr int N1 = pfa_n1(N);
  constexpr int N2 = N / N1;
  static_assert(N1 > 1 && N2 > 1 && gcd_c(N1, N2) == 1, "prime-factor split");
  cpx<T> m[N1][N2];
  static_for<0, N1>([&](auto c1) {
    static_for<0, N2>([&](auto c2) {
      constexpr int n1 = decltype(c1)::value, n2 = decltype(c2)::value;
      constexpr int src = (N2 * n1 + N1 * n2) % N;
      m[n1][n2] = a[src];
    });
  });
  static_for<0, N1>([&](auto c1) { fft<N2, DIR, T>(m[decltype(c1)::value]); });
  static_for<0, N2>([&](auto c2) {
    constexpr int k2 = decltype(c2)::value;
    cpx<T> col[N1];
    static_for<0, N1>([&](auto c1) { col[decltype(c1)::value] = m[decltype(c1)::value][k2]; });
    fft<N1, DIR, T>(col);
    static_for<0, N1>([&](auto c1) {
      constexpr int k1 = decltype(c1)::value;
      constexpr int k = crt_index(k1, k2, N1, N2);
      a[k] = col[k1];
    });
  });
}

// In-place DFT of length N on a register array: prime-factor split when N has two coprime
// factors, Cooley-Tukey otherwise.
template <int N, int DIR, typename T>
__host__ __device__ __forceinline__ void fft(cpx<T>* a) {
  static_assert(radix_ok(N), "axis length must factor into 2, 3, 5");
  if constexpr (N == 1) {
    return;
  } else if constexpr (pfa_n1(N) != 0) {
    fft_pfa<N, DIR, T>(a);
  } else {
    fft_ct<N, DIR, T>(a);
  }
}

}  // namespace hse
