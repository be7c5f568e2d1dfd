// Kernels of the size-specialised line DST (forward: FP64 block -> spectral
// scratch; inverse: spectral scratch -> block, scaled).  Included by one
// translation unit per compute precision.
#pragma once

#include "fpg_dstline.cuh"
#include "fpg_internal.cuh"

namespace fpg {
namespace dl {

// Launch shape per (compute type, p): the DFT of length p (or p - 1 under
// Rader) is A * B; Q line pairs per CTA; NT threads.
template <typename T, int P>
struct LineCfg;

#define FPG_LINECFG(TY, PP, AA, BB, RD, QQ, NTT)   \
  template <>                                      \
  struct LineCfg<TY, PP> {                         \
    static constexpr int A = AA, B = BB, Q = QQ;   \
    static constexpr int NT = NTT;                 \
    static constexpr bool rader = RD;              \
  };
FPG_LINECFG(float, 65, 13, 5, false, 16, 256)
FPG_LINECFG(float, 257, 16, 16, true, 8, 128)
FPG_LINECFG(float, 513, 27, 19, false, 8, 256)
FPG_LINECFG(float, 1025, 25, 41, false, 4, 192)
FPG_LINECFG(double, 65, 13, 5, false, 16, 256)
FPG_LINECFG(double, 257, 16, 16, true, 1, 64)
FPG_LINECFG(double, 513, 27, 19, false, 4, 128)
#undef FPG_LINECFG

// Quad form of the Rader 16 x 16 passes: each sub-DFT of length 16 is spread
// over the four lanes of a quad (4x more threads), for FP64 batches that would
// otherwise run a handful of warps per SM.
template <typename T, int P>
struct LineQuad {
  static constexpr bool value = false;
};
template <>
struct LineQuad<double, 257> {
  static constexpr bool value = true;
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

template <typename T, int P>
struct LineShape {
  using C = LineCfg<T, P>;
  static constexpr int n = P - 1;
  static constexpr int A = C::A, B = C::B, Q = C::Q, NT = C::NT;
  static constexpr bool rader = C::rader;
  static constexpr int N = A * B;             // DFT length run by the two passes
  static constexpr int YB = (B % 2 == 0) ? B + 1 : B;  // odd pitch: pass-2 reads hit distinct banks
  static constexpr int LP = n + 1;            // line pitch in shared memory (odd: column walks hit distinct banks)
  static constexpr int K = (P + 1) / 2;       // unpack terms
  static constexpr int CK = (K + 31) / 32;    // unpack terms per lane
  static_assert(N == (rader ? P - 1 : P), "plan shape");
  // shared memory, in bytes, 16-byte aligned pieces
  static constexpr size_t o_sinp = 0;  // [2][P]: sin(pi j/p) + 1/2, sin(pi j/p) - 1/2
  static constexpr size_t o_tw = align16(o_sinp + sizeof(T) * 2 * P);
  static constexpr size_t o_bhat = align16(o_tw + sizeof(C2<T>) * N);
  static constexpr size_t o_pin = align16(o_bhat + (rader ? sizeof(C2<T>) * N : 0));
  static constexpr size_t o_pout = align16(o_pin + (rader ? sizeof(int) * N : 0));
  static constexpr size_t o_dc = align16(o_pout + (rader ? sizeof(int) * N : 0));
  // x: the spectra [Q][P] (Stockham), or FFT2's pass-1 output [Q][A][YB] (Rader;
  // the final spectra then go back into y, pitch ZP)
  static constexpr int XP = (rader && A * YB > P) ? A * YB : P;
  static constexpr int ZP = rader ? A * YB : P;  // pitch of the spectra handed to unpack
  // The real lines and x share one region: the lines are dead once pass 1 has
  // packed them, and x is dead once its spectra are unpacked (non-Rader: pair q's
  // spectrum overlays pair q's two lines exactly, P = LP).  y follows.
  static constexpr size_t lines_bytes = sizeof(T) * 2 * Q * LP;
  static constexpr size_t x_bytes = sizeof(C2<T>) * Q * XP;
  static constexpr size_t o_lines = align16(o_dc + sizeof(C2<T>) * Q);
  static constexpr size_t o_x = o_lines;
  static constexpr size_t o_y = align16(o_lines + (lines_bytes > x_bytes ? lines_bytes : x_bytes));
  static constexpr size_t bytes = align16(o_y + sizeof(C2<T>) * Q * A * YB);
};

template <typename T, int P>
struct LineSmem {
  using S = LineShape<T, P>;
  T* spl;      // sin(pi j/p) + 1/2
  T* smi;      // sin(pi j/p) - 1/2
  C2<T>* tw;    // [ka][jb] = w_N^{ka jb}
  C2<T>* bhat;  // Rader kernel spectrum
  int* pin;
  int* pout;
  C2<T>* dc;
  T* lines;  // [2Q][LP] real lines (input, then output)
  C2<T>* y;  // [Q][A][YB]
  C2<T>* x;  // [Q][XP]
  __device__ __forceinline__ explicit LineSmem(unsigned char* base) {
    spl = reinterpret_cast<T*>(base + S::o_sinp);
    smi = spl + P;
    tw = reinterpret_cast<C2<T>*>(base + S::o_tw);
    bhat = reinterpret_cast<C2<T>*>(base + S::o_bhat);
    pin = reinterpret_cast<int*>(base + S::o_pin);
    pout = reinterpret_cast<int*>(base + S::o_pout);
    dc = reinterpret_cast<C2<T>*>(base + S::o_dc);
    lines = reinterpret_cast<T*>(base + S::o_lines);
    y = reinterpret_cast<C2<T>*>(base + S::o_y);
    x = reinterpret_cast<C2<T>*>(base + S::o_x);
  }
};

template <typename T, int P>
__device__ __forceinline__ void load_tables(DstPlan pl, LineSmem<T, P>& s) {
  using S = LineShape<T, P>;
  const C2<T>* W = reinterpret_cast<const C2<T>*>(pl.W);  // w_N^m, m < N
  const T* sp = reinterpret_cast<const T*>(pl.sinp);
  for (int i = threadIdx.x; i < P; i += S::NT) {
    s.spl[i] = sp[i] + T(0.5);
    s.smi[i] = sp[i] - T(0.5);
  }
  for (int i = threadIdx.x; i < S::N; i += S::NT) {
    const int ka = i / S::B, jb = i - ka * S::B;
    s.tw[i] = W[ka * jb];  // ka * jb < N
  }
  if constexpr (S::rader) {
    const C2<T>* Bh = reinterpret_cast<const C2<T>*>(pl.Bhat);
    for (int i = threadIdx.x; i < S::N; i += S::NT) {
      s.bhat[i] = Bh[i];
      s.pin[i] = pl.pin[i];
      s.pout[i] = pl.pout[i];
    }
  }
}

// (fma(cp, a1, cm a2), fma(cp, b1, cm b2)): one packed value of a line pair
template <typename T>
__device__ __forceinline__ C2<T> pack_pair(T cp, T cm, T a1, T a2, T b1, T b2) {
  if constexpr (sizeof(T) == 4) {
    const float2 t = mul2(make_float2(cm, cm), make_float2(a2, b2));
    return c2(fma2(make_float2(cp, cp), make_float2(a1, b1), t));
  } else {
    return C2<T>{fma(cp, a1, cm * a2), fma(cp, b1, cm * b2)};
  }
}

// z_j of line pair q (j in 1..p-1): u_j = sin(pi j/p)(x_j + x_{p-j}) + (x_j - x_{p-j})/2
// = (sin(pi j/p) + 1/2) x_j + (sin(pi j/p) - 1/2) x_{p-j} for the two lines,
// packed as real and imaginary part (two operations per value instead of four).
template <typename T, int P>
__device__ __forceinline__ C2<T> pack(const LineSmem<T, P>& s, int q, int j) {
  constexpr int LP = LineShape<T, P>::LP;
  const T* la = s.lines + (2 * q) * LP;
  const T* lb = la + LP;
  const T a1 = la[j - 1], a2 = la[P - j - 1], b1 = lb[j - 1], b2 = lb[P - j - 1];
  const T cp = s.spl[j], cm = s.smi[j];
  return pack_pair(cp, cm, a1, a2, b1, b2);
}

// Pass 1 of the two-pass DFT: per (pair q, jb) a DFT of length A over ja of
// in(q, B ja + jb), times w_N^{jb ka}, into y[q][ka][jb].
template <typename T, int P, typename In>
__device__ __forceinline__ void pass1(LineSmem<T, P>& s, In in) {
  using S = LineShape<T, P>;
  constexpr int A = S::A, B = S::B;
  for (int t = threadIdx.x; t < S::Q * B; t += S::NT) {
    const int q = t / B, jb = t - q * B;
    C2<T> v[A];
    static_for<A>([&](auto ja) { v[decltype(ja)::value] = in(q, B * decltype(ja)::value + jb); });
    dft<A, T>(v);
    C2<T>* yq = s.y + q * (A * S::YB) + jb;
    const C2<T>* tw = s.tw + jb;
    yq[0] = v[0];
    static_for<A - 1>([&](auto kai) {
      constexpr int ka = decltype(kai)::value + 1;
      yq[ka * S::YB] = c_mul(v[ka], tw[ka * B]);
    });
  }
}

// Pass 2: per (pair q, ka) a DFT of length B over jb of y[q][ka][jb]; output
// k = ka + A kb handed to out(q, k, value).
template <typename T, int P, typename Out>
__device__ __forceinline__ void pass2(LineSmem<T, P>& s, Out out) {
  using S = LineShape<T, P>;
  constexpr int A = S::A, B = S::B;
  for (int t = threadIdx.x; t < S::Q * A; t += S::NT) {
    const int q = t / A, ka = t - q * A;
    C2<T> v[B];
    const C2<T>* yq = s.y + q * (A * S::YB) + ka * S::YB;
    static_for<B>([&](auto jb) { v[decltype(jb)::value] = yq[decltype(jb)::value]; });
    dft<B, T>(v);
    static_for<B>([&](auto kb) { out(q, ka + A * decltype(kb)::value, v[decltype(kb)::value]); });
  }
}

template <typename T>
__device__ __forceinline__ C2<T> sel4(int i, C2<T> a0, C2<T> a1, C2<T> a2, C2<T> a3) {
  const C2<T> lo = (i & 1) ? a1 : a0, hi = (i & 1) ? a3 : a2;
  return (i & 2) ? hi : lo;
}
template <typename T>
__device__ __forceinline__ C2<T> shfl_xor_c(C2<T> v, int d) {
  return C2<T>{__shfl_xor_sync(0xffffffffu, v.x, d), __shfl_xor_sync(0xffffffffu, v.y, d)};
}
// DFT of length 16 over the four lanes of a quad, s = lane & 3: lane s holds
// x[s + 4i] in v[i] on entry and X[s + 4k] in v[k] on exit.  With j = s + 4i and
// k = k1 + 4 k2: each lane takes the DFT of length 4 over i, twiddles by
// w_16^{s k1}, the quad transposes (lane t gathers Y_s[t] from every lane s with
// three xor shuffles) and each lane takes the DFT of length 4 over s.
template <typename T>
__device__ __forceinline__ void dft16_quad(C2<T> (&v)[4], int s) {
  dft<4, T>(v);
  constexpr T c1 = (T)turn_sincos(1, 16, false), s1 = (T)turn_sincos(1, 16, true);
  constexpr T c2 = (T)turn_sincos(2, 16, false), s2 = (T)turn_sincos(2, 16, true);
  constexpr T c3 = (T)turn_sincos(3, 16, false), s3 = (T)turn_sincos(3, 16, true);
  constexpr T c6 = (T)turn_sincos(6, 16, false), s6 = (T)turn_sincos(6, 16, true);
  constexpr T c9 = (T)turn_sincos(9, 16, false), s9 = (T)turn_sincos(9, 16, true);
  const C2<T> one{T(1), T(0)};
  // w_16^{s k1} = (cos, -sin)(2 pi s k1 / 16)
  const C2<T> w1 = sel4(s, one, C2<T>{c1, -s1}, C2<T>{c2, -s2}, C2<T>{c3, -s3});
  const C2<T> w2 = sel4(s, one, C2<T>{c2, -s2}, C2<T>{T(0), T(-1)}, C2<T>{c6, -s6});
  const C2<T> w3 = sel4(s, one, C2<T>{c3, -s3}, C2<T>{c6, -s6}, C2<T>{c9, -s9});
  v[1] = c_mul(v[1], w1);
  v[2] = c_mul(v[2], w2);
  v[3] = c_mul(v[3], w3);
  const C2<T> r0 = sel4(s, v[0], v[1], v[2], v[3]);
  const C2<T> r1 = shfl_xor_c(sel4(s ^ 1, v[0], v[1], v[2], v[3]), 1);
  const C2<T> r2 = shfl_xor_c(sel4(s ^ 2, v[0], v[1], v[2], v[3]), 2);
  const C2<T> r3 = shfl_xor_c(sel4(s ^ 3, v[0], v[1], v[2], v[3]), 3);
  // u[p] = Y_p[s] came from lane p = s ^ d as r_d
  v[0] = sel4(s, r0, r1, r2, r3);
  v[1] = sel4(s ^ 1, r0, r1, r2, r3);
  v[2] = sel4(s ^ 2, r0, r1, r2, r3);
  v[3] = sel4(s ^ 3, r0, r1, r2, r3);
  dft<4, T>(v);
}

// DFT of length p of every packed line pair; returns the spectra, pair q at
// [q * ZP + k].
template <typename T, int P>
__device__ __forceinline__ const C2<T>* dft_p(LineSmem<T, P>& s) {
  using S = LineShape<T, P>;
  if constexpr (!S::rader) {
    pass1<T, P>(s, [&](int q, int j) { return j == 0 ? C2<T>{T(0), T(0)} : pack<T, P>(s, q, j); });
    __syncthreads();
    pass2<T, P>(s, [&](int q, int k, C2<T> v) { s.x[q * P + k] = v; });
    __syncthreads();
    return s.x;
  } else {
    // Rader: with g a generator mod p, A_b = z_{g^b}; X_{g^{-a}} = (A (*) w)[a],
    // w_c = w_p^{g^{-c}}, a cyclic convolution of length N = p - 1 done as
    // conj(DFT(conj(DFT(A) . B))) with B = DFT(w)/N; X_0 = sum_b A_b (z_0 = 0
    // because x_0 = x_p = 0).  N = A * A: the thread that finishes the first
    // DFT's outputs k = ka + A kb (all kb) holds exactly the inputs of the
    // second DFT's first pass for jb = ka, so the two meet in registers.
    constexpr int A = S::A, B = S::B, N = S::N, YB = S::YB;
    static_assert(A == B && N == P - 1, "Rader length A * A");
    if constexpr (LineQuad<T, P>::value) {
      static_assert(A == 16 && S::NT == S::Q * 16 * 4, "quad form: one quad per (pair, index)");
      const int sq = threadIdx.x & 3, qt = threadIdx.x >> 2;
      const int q = qt / A, g = qt - q * A;  // pass task: jb (first pass) or ka (others)
      C2<T> v[4];
      // first DFT, pass 1 (jb = g): inputs ja = sq + 4i, outputs ka = sq + 4k
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = pack<T, P>(s, q, s.pin[B * (sq + 4 * i) + g]);
      dft16_quad<T>(v, sq);
      {
        C2<T>* yq = s.y + q * (A * YB) + g;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int ka = sq + 4 * k;
          yq[ka * YB] = c_mul(v[k], s.tw[ka * B + g]);
        }
      }
      __syncthreads();
      // first DFT pass 2 (ka = g), product with B^, second DFT pass 1 (jb' = g)
      {
        const C2<T>* yq = s.y + q * (A * YB) + g * YB;
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = yq[sq + 4 * i];
        dft16_quad<T>(v, sq);  // outputs k = g + A kb, kb = sq + 4k
        if (g == 0 && sq == 0) s.dc[q] = v[0];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const C2<T> m = c_mul(v[k], s.bhat[g + A * (sq + 4 * k)]);
          v[k] = C2<T>{m.x, -m.y};
        }
        dft16_quad<T>(v, sq);  // inputs ja' = kb, outputs ka' = sq + 4k
        C2<T>* xq = s.x + q * (A * YB) + g;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int ka = sq + 4 * k;
          xq[ka * YB] = c_mul(v[k], s.tw[ka * B + g]);
        }
      }
      __syncthreads();
      // second DFT, pass 2 (ka = g); scatter X_{g^{-a}} = conj(C_a)
      {
        const C2<T>* xq = s.x + q * (A * YB) + g * YB;
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = xq[sq + 4 * i];
        dft16_quad<T>(v, sq);
        C2<T>* zq = s.y + q * S::ZP;
#pragma unroll
        for (int k = 0; k < 4; ++k) zq[s.pout[g + A * (sq + 4 * k)]] = C2<T>{v[k].x, -v[k].y};
      }
      for (int qq = threadIdx.x; qq < S::Q; qq += S::NT) s.y[qq * S::ZP] = s.dc[qq];
      __syncthreads();
      return s.y;
    }
    pass1<T, P>(s, [&](int q, int b) { return pack<T, P>(s, q, s.pin[b]); });
    __syncthreads();
    for (int t = threadIdx.x; t < S::Q * A; t += S::NT) {
      const int q = t / A, ka = t - q * A;
      C2<T> v[B];
      const C2<T>* yq = s.y + q * (A * YB) + ka * YB;
      static_for<B>([&](auto jb) { v[decltype(jb)::value] = yq[decltype(jb)::value]; });
      dft<B, T>(v);  // first DFT, outputs k = ka + A kb
      if (ka == 0) s.dc[q] = v[0];
      static_for<B>([&](auto kbi) {
        constexpr int kb = decltype(kbi)::value;
        const C2<T> m = c_mul(v[kb], s.bhat[ka + A * kb]);  // bhat carries the 1/N
        v[kb] = C2<T>{m.x, -m.y};  // conj: the inverse DFT as a forward one
      });
      // second DFT, pass 1 for jb' = ka: inputs ja' = kb are v[kb]
      dft<A, T>(v);
      C2<T>* xq = s.x + q * (A * YB) + ka;
      const C2<T>* tw = s.tw + ka;
      xq[0] = v[0];
      static_for<A - 1>([&](auto kai) {
        constexpr int kk = decltype(kai)::value + 1;
        xq[kk * YB] = c_mul(v[kk], tw[kk * B]);
      });
    }
    __syncthreads();
    // second DFT, pass 2, from x into y; scatter X_{g^{-a}} = conj(C_a)
    for (int t = threadIdx.x; t < S::Q * A; t += S::NT) {
      const int q = t / A, ka = t - q * A;
      C2<T> v[B];
      const C2<T>* xq = s.x + q * (A * YB) + ka * YB;
      static_for<B>([&](auto jb) { v[decltype(jb)::value] = xq[decltype(jb)::value]; });
      dft<B, T>(v);
      C2<T>* zq = s.y + q * S::ZP;
      static_for<B>([&](auto kbi) {
        constexpr int kb = decltype(kbi)::value;
        const C2<T> c = v[kb];
        zq[s.pout[ka + A * kb]] = C2<T>{c.x, -c.y};
      });
    }
    for (int q = threadIdx.x; q < S::Q; q += S::NT) s.y[q * S::ZP] = s.dc[q];
    __syncthreads();
    return s.y;
  }
}

// Unpack the spectra into the 2Q real output lines (in s.lines), scaled
// by 2 (the 1/2 factors are left out): for each pair, with U = (Z_k + conj Z_{p-k})/2
// (line a) and (Z_k - conj Z_{p-k})/(2i) (line b),
//   y_{2k} = -Im U_k,  y_1 = Re U_0 / 2,  y_{2k+1} = y_{2k-1} + Re U_k,
// one warp per pair, each lane a contiguous run of CK terms, a warp scan for
// the prefix sum.
template <typename T, int P>
__device__ __forceinline__ void unpack(LineSmem<T, P>& s, const C2<T>* spectra) {
  using S = LineShape<T, P>;
  constexpr int n = S::n, K = S::K, CK = S::CK;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = S::NT / 32;
  for (int q = wid; q < S::Q; q += NW) {
    const C2<T>* Z = spectra + q * S::ZP;
    T* ya = s.lines + (2 * q) * S::LP;
    T* yb = ya + S::LP;
    const int k0 = lane * CK;
    if constexpr (sizeof(T) == 4) {
      // the two lines' sums as one paired value (line a in .x, line b in .y):
      // component by component the same operations as the scalar form below
      float2 r[CK], o[CK];
      float2 sum = make_float2(0.f, 0.f);
      static_for<CK>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        const int k = k0 + i;
        r[i] = o[i] = make_float2(0.f, 0.f);
        if (k < K) {
          const float2 zk = f2(Z[k]);
          if (k == 0) {
            r[i] = zk;
          } else {
            const float2 zr = f2(Z[P - k]);
            r[i] = add2(zk, zr);
            const float2 d = add2(make_float2(zk.y, zk.x), make_float2(-zr.y, -zr.x));
            o[i] = make_float2(-d.x, d.y);
          }
          sum = add2(sum, r[i]);
        }
      });
      float2 in = sum;  // inclusive scan of the lane totals
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float2 t = make_float2(__shfl_up_sync(0xffffffffu, in.x, off), __shfl_up_sync(0xffffffffu, in.y, off));
        if (lane >= off) in = add2(in, t);
      }
      float2 acc = make_float2(__shfl_up_sync(0xffffffffu, in.x, 1), __shfl_up_sync(0xffffffffu, in.y, 1));
      if (lane == 0) acc = make_float2(0.f, 0.f);
      __syncwarp();  // the spectrum may share storage with the lines written below
      static_for<CK>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        const int k = k0 + i;
        if (k < K) {
          acc = add2(acc, r[i]);
          if (2 * k + 1 <= n) {
            ya[2 * k] = acc.x;
            yb[2 * k] = acc.y;
          }
          if (k >= 1 && 2 * k <= n) {
            ya[2 * k - 1] = o[i].x;
            yb[2 * k - 1] = o[i].y;
          }
        }
      });
    } else {
      T ra[CK], rb[CK], oa[CK], ob[CK];
      T sa = T(0), sb = T(0);
      static_for<CK>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        const int k = k0 + i;
        ra[i] = rb[i] = oa[i] = ob[i] = T(0);
        if (k < K) {
          const C2<T> zk = Z[k];
          if (k == 0) {
            ra[i] = zk.x;
            rb[i] = zk.y;
          } else {
            const C2<T> zr = Z[P - k];
            ra[i] = zk.x + zr.x;
            rb[i] = zk.y + zr.y;
            oa[i] = -(zk.y - zr.y);
            ob[i] = zk.x - zr.x;
          }
          sa += ra[i];
          sb += rb[i];
        }
      });
      T ia = sa, ib = sb;  // inclusive scan of the lane totals
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
          ia += ta;
          ib += tb;
        }
      }
      T acca = __shfl_up_sync(0xffffffffu, ia, 1), accb = __shfl_up_sync(0xffffffffu, ib, 1);
      if (lane == 0) acca = accb = T(0);
      __syncwarp();  // the spectrum may share storage with the lines written below
      static_for<CK>([&](auto ii) {
        constexpr int i = decltype(ii)::value;
        const int k = k0 + i;
        if (k < K) {
          acca += ra[i];
          accb += rb[i];
          if (2 * k + 1 <= n) {
            ya[2 * k] = acca;
            yb[2 * k] = accb;
          }
          if (k >= 1 && 2 * k <= n) {
            ya[2 * k - 1] = oa[i];
            yb[2 * k - 1] = ob[i];
          }
        }
      });
    }
  }
}

// Offset of block b of a batch (selects among the four offsets without
// indexing the parameter array, which would place it in local memory).
__device__ __forceinline__ long long boff(const BatchDesc& d, int b) {
  const int i = b % d.nper;
  const long long o = i == 0 ? d.off[0] : (i == 1 ? d.off[1] : (i == 2 ? d.off[2] : d.off[3]));
  return (long long)(b / d.nper) * d.rhs_stride + o;
}

// Forward: 2Q lines (t along the line) of block b -> DST -> scratch[b][k][s]
// (s fastest), in the compute precision, scaled by 2.
template <typename T, int P>
__global__ void __launch_bounds__(LineShape<T, P>::NT)
k_dst_lines_fwd(const double* __restrict__ in, BatchDesc ib, LineLayout L, DstPlan pl, T* __restrict__ scratch,
                const int* __restrict__ active, int nper_active, int vec) {
  using S = LineShape<T, P>;
  constexpr int n = S::n, Q = S::Q, NT = S::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  LineSmem<T, P> s(smem_raw);
  const int s0 = blockIdx.x * 2 * Q;
  const int nl = min(2 * Q, L.ns - s0);
  load_tables<T, P>(pl, s);
  const double* src = in + boff(ib, b);
  constexpr int LP = S::LP;
  if (vec) {  // rows contiguous (st == 1) and 16-byte aligned: two values per load
    // U loads in flight per thread before any is converted and stored
    constexpr int U = 8;
    for (int i0 = threadIdx.x; i0 < Q * n; i0 += NT * U) {
      double2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * NT;
        const int l = i / (n / 2), t2 = i - l * (n / 2);
        v[u] = make_double2(0.0, 0.0);
        if (i < Q * n && l < nl) v[u] = *reinterpret_cast<const double2*>(src + (long long)(s0 + l) * L.ss + 2 * t2);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * NT;
        if (i < Q * n) {
          const int l = i / (n / 2), t2 = i - l * (n / 2);
          s.lines[l * LP + 2 * t2] = convert<T>(v[u].x);
          s.lines[l * LP + 2 * t2 + 1] = convert<T>(v[u].y);
        }
      }
    }
  } else {
    for (int i = threadIdx.x; i < 2 * Q * n; i += NT) {
      const int l = i / n, t = i - l * n;
      const double v = l < nl ? src[(long long)t * L.st + (long long)(s0 + l) * L.ss] : 0.0;
      s.lines[l * LP + t] = convert<T>(v);
    }
  }
  __syncthreads();
  unpack<T, P>(s, dft_p<T, P>(s));
  __syncthreads();
  // scratch[b][k][s]: rows l fastest, a warp writes runs of nl consecutive rows
  T* dst = scratch + (long long)b * n * L.ns + s0;
  for (int i = threadIdx.x; i < nl * n; i += NT) {
    const int k = i / nl, l = i - k * nl;
    dst[(long long)k * L.ns + l] = s.lines[l * LP + k];
  }
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (cp.async.bulk, completion counted on an mbarrier).

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous transfer, then the copy
// of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global memory.
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, unsigned bytes, unsigned long long* mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(sdst)),
               "l"(gsrc), "r"(bytes), "r"(smem_addr(mbar))
               : "memory");
}

// Wait for phase `parity` of the barrier; false after `limit` unsuccessful tries.
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <typename T, int P>
struct BulkShape {
  using S = LineShape<T, P>;
  static constexpr size_t o_stage = align16(S::bytes);
  static constexpr size_t o_mbar = align16(o_stage + sizeof(double) * 2 * S::Q * S::n);
  static constexpr size_t bytes = o_mbar + 16;
};

// Persistent form of the forward DST for blocks whose lines are contiguous rows
// (st == 1, ss == n, 16-byte aligned): each CTA walks the tiles (2Q lines of one
// block) blockIdx.x, blockIdx.x + gridDim.x, ...; thread 0 fetches the next
// tile's FP64 rows with one bulk copy into a staging buffer as soon as the
// current tile has been converted out of it, so the load overlaps the current
// tile's transform.  Thread 0 waits for each copy, at most `wait_limit` tries
// (0: gives up at once), and tells the CTA through shared memory, so every
// thread takes the same branch.  A wait that runs out sets *err = 1; thread 0
// then waits (again bounded) for the copy in flight to land, and the whole CTA
// returns: no trap, nothing left writing into freed shared memory.
template <typename T, int P>
__global__ void __launch_bounds__(LineShape<T, P>::NT)
k_dst_lines_fwd_bulk(const double* __restrict__ in, BatchDesc ib, LineLayout L, DstPlan pl, T* __restrict__ scratch,
                     const int* __restrict__ active, int nper_active, int nblk, int* __restrict__ err,
                     int wait_limit) {
  using S = LineShape<T, P>;
  using BS = BulkShape<T, P>;
  constexpr int n = S::n, Q = S::Q, NT = S::NT, LP = S::LP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LineSmem<T, P> s(smem_raw);
  double* stage = reinterpret_cast<double*>(smem_raw + BS::o_stage);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem_raw + BS::o_mbar);
  __shared__ int s_landed;
  const int tpb = (L.ns + 2 * Q - 1) / (2 * Q);
  const int total = nblk * tpb;
  auto live = [&](int tile) { return active == nullptr || active[(tile / tpb) / nper_active]; };
  auto next_of = [&](int tile) {
    do tile += gridDim.x;
    while (tile < total && !live(tile));
    return tile;
  };
  auto issue = [&](int tile) {
    const int b = tile / tpb, s0 = (tile - b * tpb) * 2 * Q;
    const int nl = min(2 * Q, L.ns - s0);
    bulk_load(stage, in + boff(ib, b) + (long long)s0 * n, (unsigned)(nl * n * sizeof(double)), mbar);
  };
  if (threadIdx.x == 0) mbar_init(mbar, 1);
  load_tables<T, P>(pl, s);
  __syncthreads();
  int tile = blockIdx.x;
  if (tile < total && !live(tile)) tile = next_of(tile);
  if (threadIdx.x == 0 && tile < total) issue(tile);
  unsigned parity = 0;
  while (tile < total) {
    const int b = tile / tpb, s0 = (tile - b * tpb) * 2 * Q;
    const int nl = min(2 * Q, L.ns - s0);
    if (threadIdx.x == 0) s_landed = mbar_wait(mbar, parity, wait_limit) ? 1 : 0;
    __syncthreads();
    if (!s_landed) {  // the same value in every thread
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        mbar_wait(mbar, parity, 1 << 20);  // the copy in flight lands before the CTA leaves
      }
      return;
    }
    mbar_wait(mbar, parity, 1 << 22);  // phase complete: returns at once, and orders the copied data
    parity ^= 1u;
    for (int i = threadIdx.x; i < 2 * Q * n; i += NT) {
      const int l = i / n, tt = i - l * n;
      s.lines[l * LP + tt] = l < nl ? convert<T>(stage[i]) : T(0);
    }
    __syncthreads();  // the staging buffer is free
    const int next = next_of(tile);
    if (threadIdx.x == 0 && next < total) issue(next);
    unpack<T, P>(s, dft_p<T, P>(s));
    __syncthreads();
    T* dst = scratch + (long long)b * n * L.ns + s0;
    for (int i = threadIdx.x; i < nl * n; i += NT) {
      const int k = i / nl, l = i - k * nl;
      dst[(long long)k * L.ns + l] = s.lines[l * LP + k];
    }
    __syncthreads();  // lines are rewritten by the next tile's conversion
    tile = next;
  }
}

// ---------------------------------------------------------------------------
// Streaming persistent forward DST (FP32 compute; p without Rader; tiles of 2Q
// contiguous, 16-byte aligned rows, ns a multiple of 2Q).  Same arithmetic in the
// same order as k_dst_lines_fwd, so the output is bit-identical; what changes is
// the movement of data:
//   * each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... and keeps the
//     packing and twiddle tables in shared memory for all of them;
//   * the next tile's FP64 rows arrive by one bulk copy (cp.async.bulk on an
//     mbarrier) into a staging buffer while the current tile is transformed;
//   * the packing reads the staging buffer directly: one pair of loads x_{j-1},
//     x_{p-j-1} gives both u_j and u_{p-j} (sin(pi (p-j)/p) = sin(pi j/p)), so the
//     real lines never pass through shared memory in FP32;
//   * both passes of the DFT and the unpacking run in place in one buffer of Q
//     spectra (each pass reads its inputs into registers, the CTA synchronises, then
//     writes), which with the staging buffer leaves two CTAs per SM;
//   * the transposed store to scratch[b][k][s] writes runs of 2Q rows as float4.
template <int P>
struct StreamShape {
  using S = LineShape<float, P>;
  static constexpr int n = S::n, Q = S::Q;
  static constexpr size_t o_spl = 0;                                   // [P] sin(pi j/p) + 1/2
  static constexpr size_t o_smi = align16(o_spl + sizeof(float) * P);  // [P] sin(pi j/p) - 1/2
  static constexpr size_t o_tw = align16(o_smi + sizeof(float) * P);   // [N] w_p^{ka jb}
  static constexpr size_t o_z = align16(o_tw + sizeof(C2<float>) * S::N);
  static constexpr size_t o_stage = align16(o_z + sizeof(C2<float>) * Q * P);
  static constexpr size_t o_mbar = align16(o_stage + sizeof(double) * 2 * Q * n);
  static constexpr size_t bytes = o_mbar + 16;
  static constexpr bool eligible = !S::rader && S::YB == S::B && S::ZP == P && S::LP == P &&
                                   Q * S::B <= S::NT && Q * S::A <= S::NT && (2 * Q) % 4 == 0;
};

template <int P>
__global__ void __launch_bounds__(LineShape<float, P>::NT, 2)
k_dst_lines_fwd_stream(const double* __restrict__ in, BatchDesc ib, LineLayout L, DstPlan pl,
                       float* __restrict__ scratch, const int* __restrict__ active, int nper_active, int nblk,
                       int* __restrict__ err, int wait_limit) {
  using T = float;
  using S = LineShape<T, P>;
  using SS = StreamShape<P>;
  static_assert(SS::eligible, "streaming forward DST: non-Rader p with in-place passes");
  constexpr int n = S::n, Q = S::Q, NT = S::NT, A = S::A, B = S::B, YB = S::YB, N = S::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* spl = reinterpret_cast<T*>(smem_raw + SS::o_spl);
  T* smi = reinterpret_cast<T*>(smem_raw + SS::o_smi);
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw + SS::o_tw);
  C2<T>* Z = reinterpret_cast<C2<T>*>(smem_raw + SS::o_z);
  double* stage = reinterpret_cast<double*>(smem_raw + SS::o_stage);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem_raw + SS::o_mbar);
  __shared__ int s_landed;
  // the unpacking writes the 2Q real lines over the Q spectra (pitch LP = P)
  LineSmem<T, P> ls(smem_raw);
  ls.lines = reinterpret_cast<T*>(Z);
  const int tpb = L.ns / (2 * Q);
  const int total = nblk * tpb;
  auto live = [&](int tile) { return active == nullptr || active[(tile / tpb) / nper_active]; };
  auto next_of = [&](int tile) {
    do tile += gridDim.x;
    while (tile < total && !live(tile));
    return tile;
  };
  auto issue = [&](int tile) {
    const int b = tile / tpb, s0 = (tile - b * tpb) * 2 * Q;
    bulk_load(stage, in + boff(ib, b) + (long long)s0 * n, (unsigned)(2 * Q * n * sizeof(double)), mbar);
  };
  if (threadIdx.x == 0) mbar_init(mbar, 1);
  {
    const C2<T>* W = reinterpret_cast<const C2<T>*>(pl.W);
    const T* sp = reinterpret_cast<const T*>(pl.sinp);
    for (int i = threadIdx.x; i < P; i += NT) {
      spl[i] = sp[i] + T(0.5);
      smi[i] = sp[i] - T(0.5);
    }
    for (int i = threadIdx.x; i < N; i += NT) {
      const int ka = i / B, jb = i - ka * B;
      tw[i] = W[ka * jb];
    }
  }
  __syncthreads();
  int tile = blockIdx.x;
  if (tile < total && !live(tile)) tile = next_of(tile);
  if (threadIdx.x == 0 && tile < total) issue(tile);
  // this thread's tasks in the two passes, the same for every tile
  const int t = threadIdx.x;
  const int q1 = t / B, jb1 = t - q1 * B;  // pass 1 (t < Q B)
  const int q2 = t / A, ka2 = t - q2 * A;  // pass 2 (t < Q A)
  unsigned parity = 0;
  while (tile < total) {
    const int b = tile / tpb, s0 = (tile - b * tpb) * 2 * Q;
    if (t == 0) s_landed = mbar_wait(mbar, parity, wait_limit) ? 1 : 0;
    __syncthreads();
    if (!s_landed) {  // the same value in every thread
      if (t == 0) {
        atomicExch(err, 1);
        mbar_wait(mbar, parity, 1 << 20);  // the copy in flight lands before the CTA leaves
      }
      return;
    }
    mbar_wait(mbar, parity, 1 << 22);  // phase complete: returns at once, and orders the copied data
    parity ^= 1u;
    // packing straight from the FP64 rows: z_j and z_{p-j} of pair q
#pragma unroll 2
    for (int i = t; i < Q * (n / 2); i += NT) {
      const int q = i / (n / 2), j = i - q * (n / 2) + 1;
      const double* ra = stage + (2 * q) * n;
      const double* rb = ra + n;
      const T a1 = f64_to_f32(ra[j - 1]), a2 = f64_to_f32(ra[P - j - 1]);
      const T b1 = f64_to_f32(rb[j - 1]), b2 = f64_to_f32(rb[P - j - 1]);
      const T cp = spl[j], cm = smi[j];
      Z[q * P + j] = pack_pair(cp, cm, a1, a2, b1, b2);
      Z[q * P + P - j] = pack_pair(cp, cm, a2, a1, b2, b1);
    }
    if (t < Q) Z[t * P] = C2<T>{T(0), T(0)};
    __syncthreads();  // the staging buffer is free
    const int next = next_of(tile);
    if (t == 0 && next < total) issue(next);
    {  // pass 1: per (q, jb) a DFT of length A over ja, times w_p^{jb ka}, in place
      C2<T> v[A];
      if (t < Q * B) static_for<A>([&](auto ja) { v[decltype(ja)::value] = Z[q1 * P + B * decltype(ja)::value + jb1]; });
      __syncthreads();
      if (t < Q * B) {
        dft<A, T>(v);
        C2<T>* yq = Z + q1 * P + jb1;
        yq[0] = v[0];
        static_for<A - 1>([&](auto kai) {
          constexpr int ka = decltype(kai)::value + 1;
          yq[ka * YB] = c_mul(v[ka], tw[ka * B + jb1]);
        });
      }
      __syncthreads();
    }
    {  // pass 2: per (q, ka) a DFT of length B over jb, output k = ka + A kb, in place
      C2<T> u[B];
      if (t < Q * A) static_for<B>([&](auto jb) { u[decltype(jb)::value] = Z[q2 * P + ka2 * YB + decltype(jb)::value]; });
      __syncthreads();
      if (t < Q * A) {
        dft<B, T>(u);
        static_for<B>([&](auto kb) { Z[q2 * P + ka2 + A * decltype(kb)::value] = u[decltype(kb)::value]; });
      }
      __syncthreads();
    }
    unpack<T, P>(ls, Z);
    __syncthreads();
    // scratch[b][k][s]: runs of 2Q rows, four rows per store
    T* dst = scratch + (long long)b * n * L.ns + s0;
    constexpr int R4 = 2 * Q / 4;
#pragma unroll 2
    for (int i = t; i < n * R4; i += NT) {
      const int k = i / R4, l = (i - k * R4) * 4;
      const T* col = ls.lines + k;
      *reinterpret_cast<float4*>(dst + (long long)k * L.ns + l) =
          make_float4(col[l * P], col[(l + 1) * P], col[(l + 2) * P], col[(l + 3) * P]);
    }
    __syncthreads();  // the spectra buffer is rewritten by the next tile's packing
    tile = next;
  }
}

template <int P>
cudaError_t fwd_stream_one(const double* in, BatchDesc ib, LineLayout L, const DstPlan& pl, float* scratch, int nblk,
                           const int* active, int nper_active, int* err, int wait_limit, cudaStream_t st) {
  if constexpr (!StreamShape<P>::eligible) {
    return cudaErrorNotSupported;
  } else {
    using S = LineShape<float, P>;
    using SS = StreamShape<P>;
    static PerDeviceOnce attr;
    static int per_sm_of[64] = {};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    int per_sm = 0;
    if (auto once = attr.first()) {  // the occupancy is recorded before the device is marked done
      cudaFuncSetAttribute(k_dst_lines_fwd_stream<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS::bytes);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dst_lines_fwd_stream<P>, S::NT, SS::bytes);
      if (per_sm < 1) per_sm = 1;
      if (dev >= 0 && dev < 64) per_sm_of[dev] = per_sm;
    } else if (dev >= 0 && dev < 64) {
      per_sm = per_sm_of[dev];
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)nblk * (L.ns / (2 * S::Q));
    const int grid = (int)(total < (long long)per_sm * sms ? total : (long long)per_sm * sms);
    if (grid <= 0) return cudaSuccess;
    k_dst_lines_fwd_stream<P><<<grid, S::NT, SS::bytes, st>>>(in, ib, L, pl, scratch, active, nper_active, nblk, err,
                                                              wait_limit);
    return cudaGetLastError();
  }
}

// Inverse: scratch[b][k][s] -> DST -> out block (To), times `scale`.
template <typename T, typename To, int P>
__global__ void __launch_bounds__(LineShape<T, P>::NT)
k_dst_lines_inv(const T* __restrict__ scratch, To* __restrict__ out, BatchDesc ob, LineLayout L, DstPlan pl, T scale,
                const int* __restrict__ active, int nper_active, int vec) {
  using S = LineShape<T, P>;
  constexpr int n = S::n, Q = S::Q, NT = S::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.y;
  if (active != nullptr && !active[b / nper_active]) return;
  LineSmem<T, P> s(smem_raw);
  const int s0 = blockIdx.x * 2 * Q;
  const int nl = min(2 * Q, L.ns - s0);
  load_tables<T, P>(pl, s);
  constexpr int LP = S::LP;
  const T* src = scratch + (long long)b * n * L.ns + s0;  // [b][k][s]
  {
    constexpr int U = 8;  // loads in flight per thread
    for (int i0 = threadIdx.x; i0 < 2 * Q * n; i0 += NT * U) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * NT;
        const int k = i / (2 * Q), l = i - k * (2 * Q);
        v[u] = (i < 2 * Q * n && l < nl) ? src[(long long)k * L.ns + l] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * NT;
        if (i < 2 * Q * n) {
          const int k = i / (2 * Q), l = i - k * (2 * Q);
          s.lines[l * LP + k] = v[u];
        }
      }
    }
  }
  __syncthreads();
  unpack<T, P>(s, dft_p<T, P>(s));
  __syncthreads();
  To* dst = out + boff(ob, b);
  if (vec) {  // rows contiguous and aligned for two-element stores
    for (int i = threadIdx.x; i < nl * (n / 2); i += NT) {
      const int l = i / (n / 2), t2 = i - l * (n / 2);
      const To a = convert<To>(s.lines[l * LP + 2 * t2] * scale);
      const To c = convert<To>(s.lines[l * LP + 2 * t2 + 1] * scale);
      To* d = dst + (long long)(s0 + l) * L.ss + 2 * t2;
      if constexpr (sizeof(To) == 8) {
        *reinterpret_cast<double2*>(d) = make_double2(a, c);
      } else {
        *reinterpret_cast<float2*>(d) = make_float2(a, c);
      }
    }
  } else {
    for (int i = threadIdx.x; i < nl * n; i += NT) {
      const int l = i / n, k = i - l * n;
      dst[(long long)k * L.st + (long long)(s0 + l) * L.ss] = convert<To>(s.lines[l * LP + k] * scale);
    }
  }
}

// Host side --------------------------------------------------------------------

template <typename T, int P>
cudaError_t fwd_one(const double* in, BatchDesc ib, LineLayout L, const DstPlan& pl, T* scratch, int nblk,
                    const int* active, int nper_active, int vec, cudaStream_t st) {
  using S = LineShape<T, P>;
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_dst_lines_fwd<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
  }
  dim3 grid((L.ns + 2 * S::Q - 1) / (2 * S::Q), nblk);
  k_dst_lines_fwd<T, P><<<grid, S::NT, S::bytes, st>>>(in, ib, L, pl, scratch, active, nper_active, vec);
  return cudaGetLastError();
}

template <typename T, int P>
cudaError_t fwd_bulk_one(const double* in, BatchDesc ib, LineLayout L, const DstPlan& pl, T* scratch, int nblk,
                         const int* active, int nper_active, int* err, int wait_limit, cudaStream_t st) {
  using S = LineShape<T, P>;
  using BS = BulkShape<T, P>;
  static PerDeviceOnce attr;
  static int per_sm_of[64] = {};
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  int per_sm = 0;
  if (auto once = attr.first()) {  // the occupancy is recorded before the device is marked done
    cudaFuncSetAttribute(k_dst_lines_fwd_bulk<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BS::bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dst_lines_fwd_bulk<T, P>, S::NT, BS::bytes);
    if (per_sm < 1) per_sm = 1;
    if (dev >= 0 && dev < 64) per_sm_of[dev] = per_sm;
  } else if (dev >= 0 && dev < 64) {
    per_sm = per_sm_of[dev];
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tpb = (L.ns + 2 * S::Q - 1) / (2 * S::Q);
  const long long total = (long long)nblk * tpb;
  const int grid = (int)(total < (long long)per_sm * sms ? total : (long long)per_sm * sms);
  k_dst_lines_fwd_bulk<T, P><<<grid, S::NT, BS::bytes, st>>>(in, ib, L, pl, scratch, active, nper_active, nblk, err,
                                                              wait_limit);
  return cudaGetLastError();
}

template <typename T, typename To, int P>
cudaError_t inv_one(const T* scratch, To* out, BatchDesc ob, LineLayout L, const DstPlan& pl, int nblk,
                    const int* active, int nper_active, int vec, cudaStream_t st) {
  using S = LineShape<T, P>;
  static PerDeviceOnce attr;
  if (auto once = attr.first()) {
    cudaFuncSetAttribute(k_dst_lines_inv<T, To, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
  }
  // 2/p for the normalisation, 1/4 for the two left-out factors 1/2 (exact)
  const T scale = (T(2) / T(P)) * T(0.25);
  dim3 grid((L.ns + 2 * S::Q - 1) / (2 * S::Q), nblk);
  k_dst_lines_inv<T, To, P><<<grid, S::NT, S::bytes, st>>>(scratch, out, ob, L, pl, scale, active, nper_active, vec);
  return cudaGetLastError();
}

}  // namespace dl
}  // namespace fpg
