// Size-specialised DST-I of many lines (the hot transform of the fast solve,
// Sec. 2.1, Eq. "Dirichlet_mat_decomp": the paper applies Q through an FFT).
//
// Same mathematics as the generic engine (two real lines packed into one
// complex sequence of length p = n + 1, one complex DFT of length p, unpacking
// with a prefix sum), but every length, radix and index is a compile-time
// constant, and the DFT of length p = A * B is done in two passes over shared
// memory ("four-step" Cooley-Tukey), each thread computing one whole DFT of
// length A (pass 1) or B (pass 2) in registers:
//   j = B ja + jb,  k = ka + A kb,
//   pass 1 (per jb):  Y[jb][ka] = w_p^{jb ka} sum_ja z[B ja + jb] w_A^{ja ka}
//   pass 2 (per ka):  X[ka + A kb] = sum_jb Y[jb][ka] w_B^{jb kb}.
// A prime p (257) goes through Rader's algorithm: a cyclic convolution of
// length p - 1 = 16 * 16 done with two such two-pass FFTs.  The register DFTs
// use constants folded at compile time; composite sub-lengths (16, 25, 27) are
// split once more inside the registers.
//
// Scaling: the 1/2 factors of the unpacking step are left out (they are exact
// powers of two); the caller folds a factor 4 into the final 2/p scaling, which
// gives bit-identical results.
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "fpg_dst.cuh"

namespace fpg {
namespace dl {

// ---------------------------------------------------------------------------
// Compile-time loops and constants.

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// sin and cos of 2 pi m / R, evaluated by the compiler: the fraction m / R is
// reduced exactly to one octant, where a Taylor series of 14 terms is accurate
// to double rounding.
constexpr double kQuarterPi = 0.78539816339744830961566084581987572;

__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
// want_sin: sin(2 pi m / R), else cos(2 pi m / R).
__host__ __device__ constexpr double turn_sincos(long long m, long long R, bool want_sin) {
  m %= R;
  if (m < 0) m += R;
  const long long oct = (8 * m) / R;
  const long long rem = 8 * m - oct * R;  // angle = pi/4 (oct + rem / R)
  const bool odd = (oct & 1) != 0;
  const double x = kQuarterPi * (double)(odd ? R - rem : rem) / (double)R;
  const double s = taylor_sin(x), c = taylor_cos(x);
  double sn = 0.0, cs = 0.0;
  switch (oct) {
    case 0: sn = s; cs = c; break;
    case 1: sn = c; cs = s; break;
    case 2: sn = c; cs = -s; break;
    case 3: sn = s; cs = -c; break;
    case 4: sn = -s; cs = -c; break;
    case 5: sn = -c; cs = -s; break;
    case 6: sn = -c; cs = s; break;
    default: sn = -s; cs = c; break;
  }
  return want_sin ? sn : cs;
}

// FP32 complex arithmetic runs on the paired FP32 instructions (FADD2, FMUL2,
// FFMA2: two lanes of binary32 per instruction, each rounded exactly as the
// scalar operation).  Every paired form below computes, component by component,
// the same operations in the same order as the scalar form next to it, so the
// results are bit-identical; the transforms are issue-bound and the pairing
// halves their floating-point instruction count.
__device__ __forceinline__ float2 f2(C2<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ C2<float> c2(float2 a) { return C2<float>{a.x, a.y}; }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ C2<T> c_add(C2<T> a, C2<T> b) {
  if constexpr (sizeof(T) == 4) {
    return c2(add2(f2(a), f2(b)));
  } else {
    return C2<T>{a.x + b.x, a.y + b.y};
  }
}
template <typename T>
__device__ __forceinline__ C2<T> c_sub(C2<T> a, C2<T> b) {
  if constexpr (sizeof(T) == 4) {
    return c2(add2(f2(a), make_float2(-b.x, -b.y)));  // a + (-b) = a - b exactly
  } else {
    return C2<T>{a.x - b.x, a.y - b.y};
  }
}
template <typename T>
__device__ __forceinline__ C2<T> c_mul(C2<T> a, C2<T> w) {
  if constexpr (sizeof(T) == 4) {
    // (fma(a.x, w.x, -(a.y w.y)), fma(a.x, w.y, a.y w.x))
    const float2 t = mul2(make_float2(a.y, a.y), make_float2(w.y, w.x));
    return c2(fma2(make_float2(a.x, a.x), make_float2(w.x, w.y), make_float2(-t.x, t.y)));
  } else {
    return C2<T>{fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x)};
  }
}

// a * w_R^M with w_R = exp(-2 pi i / R), M and R compile-time.
template <int M, int R, typename T>
__device__ __forceinline__ C2<T> c_mul_root(C2<T> a) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (2 * m == R) {
    return C2<T>{-a.x, -a.y};
  } else if constexpr (4 * m == R) {  // -i
    return C2<T>{a.y, -a.x};
  } else if constexpr (4 * m == 3 * R) {  // +i
    return C2<T>{-a.y, a.x};
  } else {
    constexpr T c = (T)turn_sincos(m, R, false);
    constexpr T s = (T)turn_sincos(m, R, true);
    // (a.x + i a.y)(c - i s)
    if constexpr (sizeof(T) == 4) {
      // (fma(a.x, c, a.y s), fma(a.y, c, -(a.x s)))
      const float2 t = mul2(make_float2(a.y, a.x), make_float2(s, s));
      return c2(fma2(make_float2(a.x, a.y), make_float2(c, c), make_float2(t.x, -t.y)));
    } else {
      return C2<T>{fma(a.x, c, a.y * s), fma(a.y, c, -(a.x * s))};
    }
  }
}

// ---------------------------------------------------------------------------
// DFT (forward sign) of R values held in registers, natural order in and out.

template <int R>
struct IsPrime {
  static constexpr bool value = [] {
    if (R < 2) return false;
    for (int d = 2; d * d <= R; ++d)
      if (R % d == 0) return false;
    return true;
  }();
};

template <int R, typename T>
__device__ __forceinline__ void dft(C2<T> (&v)[R]);

// Odd prime R: pair q with R - q.  With s_q = v_q + v_{R-q}, d_q = v_q - v_{R-q},
// X_k = v_0 + sum_q s_q cos(2 pi q k / R) - i sum_q d_q sin(2 pi q k / R) and
// X_{R-k} its counterpart with +i.
template <int R, typename T>
__device__ __forceinline__ void dft_odd_prime(C2<T> (&v)[R]) {
  constexpr int H = (R - 1) / 2;
  C2<T> s[H], d[H];
  C2<T> x0 = v[0];
  static_for<H>([&](auto qi) {
    constexpr int q = decltype(qi)::value + 1;
    s[q - 1] = c_add(v[q], v[R - q]);
    d[q - 1] = c_sub(v[q], v[R - q]);
    x0 = c_add(x0, s[q - 1]);
  });
  C2<T> out[R];
  out[0] = x0;
  static_for<H>([&](auto ki) {
    constexpr int k = decltype(ki)::value + 1;
    if constexpr (sizeof(T) == 4) {
      float2 a2 = f2(v[0]), b2 = make_float2(0.f, 0.f);
      static_for<H>([&](auto qi) {
        constexpr int q = decltype(qi)::value + 1;
        constexpr int m = (q * k) % R;
        constexpr float c = (float)turn_sincos(m, R, false);
        constexpr float sn = (float)turn_sincos(m, R, true);
        a2 = fma2(f2(s[q - 1]), make_float2(c, c), a2);
        b2 = fma2(f2(d[q - 1]), make_float2(sn, sn), b2);
      });
      out[k] = c2(add2(a2, make_float2(b2.y, -b2.x)));      // a - i b
      out[R - k] = c2(add2(a2, make_float2(-b2.y, b2.x)));  // a + i b
    } else {
      C2<T> a = v[0], b{T(0), T(0)};
      static_for<H>([&](auto qi) {
        constexpr int q = decltype(qi)::value + 1;
        constexpr int m = (q * k) % R;
        constexpr T c = (T)turn_sincos(m, R, false);
        constexpr T sn = (T)turn_sincos(m, R, true);
        a.x = fma(s[q - 1].x, c, a.x);
        a.y = fma(s[q - 1].y, c, a.y);
        b.x = fma(d[q - 1].x, sn, b.x);
        b.y = fma(d[q - 1].y, sn, b.y);
      });
      out[k] = C2<T>{a.x + b.y, a.y - b.x};      // a - i b
      out[R - k] = C2<T>{a.x - b.y, a.y + b.x};  // a + i b
    }
  });
  static_for<R>([&](auto i) { v[decltype(i)::value] = out[decltype(i)::value]; });
}

// R = R1 * R2 in registers: j = R2 ja + jb, k = ka + R1 kb.
template <int R1, int R2, typename T>
__device__ __forceinline__ void dft_split(C2<T> (&v)[R1 * R2]) {
  constexpr int R = R1 * R2;
  C2<T> t[R];
  static_for<R2>([&](auto jbi) {
    constexpr int jb = decltype(jbi)::value;
    C2<T> u[R1];
    static_for<R1>([&](auto jai) { u[decltype(jai)::value] = v[R2 * decltype(jai)::value + jb]; });
    dft<R1, T>(u);
    static_for<R1>([&](auto kai) {
      constexpr int ka = decltype(kai)::value;
      t[jb * R1 + ka] = c_mul_root<jb * ka, R, T>(u[ka]);
    });
  });
  static_for<R1>([&](auto kai) {
    constexpr int ka = decltype(kai)::value;
    C2<T> u[R2];
    static_for<R2>([&](auto jbi) { u[decltype(jbi)::value] = t[decltype(jbi)::value * R1 + ka]; });
    dft<R2, T>(u);
    static_for<R2>([&](auto kbi) { v[ka + R1 * decltype(kbi)::value] = u[decltype(kbi)::value]; });
  });
}

template <int R, typename T>
__device__ __forceinline__ void dft(C2<T> (&v)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    const C2<T> a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
  } else if constexpr (R == 4) {
    const C2<T> t0 = c_add(v[0], v[2]), t1 = c_sub(v[0], v[2]);
    const C2<T> t2 = c_add(v[1], v[3]), dd = c_sub(v[1], v[3]);
    const C2<T> t3{dd.y, -dd.x};  // -i (v1 - v3)
    v[0] = c_add(t0, t2);
    v[1] = c_add(t1, t3);
    v[2] = c_sub(t0, t2);
    v[3] = c_sub(t1, t3);
  } else if constexpr (IsPrime<R>::value) {
    dft_odd_prime<R, T>(v);
  } else if constexpr (R % 4 == 0) {
    dft_split<4, R / 4, T>(v);
  } else if constexpr (R % 3 == 0) {
    dft_split<3, R / 3, T>(v);
  } else if constexpr (R % 5 == 0) {
    dft_split<5, R / 5, T>(v);
  } else {
    static_assert(R % 2 == 0, "unsupported register DFT length");
    dft_split<2, R / 2, T>(v);
  }
}

// ---------------------------------------------------------------------------
// Integer-pipe conversions between binary64 and binary32.  On this GPU the
// hardware conversion runs on the FP64 pipe (a few results per SM and clock);
// these work on the IEEE-754 encodings with 32-bit integer operations.

// binary64 -> binary32, round to nearest even.  Magnitudes below 2^-126 give a
// signed zero (no binary32 subnormals); 2^128 and above, inf and NaN give inf.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u, ahi = hi & 0x7fffffffu;
  // exponent rebiased 1023 -> 127 at bits 30..23, top 23 mantissa bits below
  unsigned em = ((ahi - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  em += (unsigned)(rest > 0x10000000u) | ((unsigned)(rest == 0x10000000u) & em);
  em = ahi < (897u << 20) ? 0u : em;
  em = ahi >= (1151u << 20) ? 0x7f800000u : em;
  return __uint_as_float(sign | em);
}

// binary32 -> binary64, exact for normal numbers, zeros, inf and NaN;
// binary32 subnormals give a signed zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, a = u & 0x7fffffffu;
  unsigned hi = sign | ((a >> 3) + (896u << 20));
  unsigned lo = a << 29;
  if (a < 0x00800000u) {
    hi = sign;
    lo = 0u;
  } else if (a >= 0x7f800000u) {
    hi = sign | 0x7ff00000u | (a > 0x7f800000u ? 0x00080000u : 0u);
    lo = 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

template <typename To, typename From>
__device__ __forceinline__ To convert(From v) {
  if constexpr (sizeof(To) == sizeof(From)) {
    return (To)v;
  } else if constexpr (sizeof(To) == 4) {
    return f64_to_f32((double)v);
  } else {
    return f32_to_f64((float)v);
  }
}

}  // namespace dl

// One Stockham stage of radix R in {2, 4, 8, 16} with the register DFT of
// length R (constants folded at compile time); otherwise as stockham_stage.
template <int R, typename T>
__device__ __forceinline__ void stockham_stage_pow2(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, int Q,
                                                    int N, int Ns, int pitch, const C2<T>* __restrict__ W) {
  const int nb = N / R;
  const int tstep = N / (Ns * R);
  for (int idx = threadIdx.x; idx < Q * nb; idx += blockDim.x) {
    const int q = idx / nb, j = idx - q * nb;
    const C2<T>* a = in + q * pitch;
    const int jm = j % Ns;
    C2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[j + r * nb];
    if (jm != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], W[jm * r * tstep]);
    }
    dl::dft<R, T>(v);
    C2<T>* o = out + q * pitch + (j - jm) * R + jm;
#pragma unroll
    for (int k = 0; k < R; ++k) o[k * Ns] = v[k];
  }
}

template <typename T>
__device__ void stockham_pow2(int R, const C2<T>* in, C2<T>* out, int Q, int N, int Ns, int pitch,
                              const C2<T>* W) {
  switch (R) {
    case 2: stockham_stage_pow2<2, T>(in, out, Q, N, Ns, pitch, W); break;
    case 4: stockham_stage_pow2<4, T>(in, out, Q, N, Ns, pitch, W); break;
    case 8: stockham_stage_pow2<8, T>(in, out, Q, N, Ns, pitch, W); break;
    default: stockham_stage_pow2<16, T>(in, out, Q, N, Ns, pitch, W); break;  // plans hold 2, 4, 8, 16 only
  }
}

}  // namespace fpg
