// FFT-based DST-I of many lines at once, inside one CTA's shared memory.
//
// DST-I_n(x)_k = sum_{t=1..n} x_t sin(pi t k / p), p = n + 1 (the unnormalised
// form of Q_D, Eq. "eigvector_Diri"; the paper computes Q p through an FFT,
// Eq. "Dirichlet_mat_decomp").  Route taken here, for p of any size:
//   * two real lines a, b are packed into one complex sequence of length p,
//       z_j = u^a_j + i u^b_j,  u_j = sin(pi j/p)(x_j + x_{p-j}) + (x_j - x_{p-j})/2,
//     with x_0 = x_p = 0;
//   * Z = DFT_p(z) by a mixed-radix Stockham FFT (radices 2, 4 and odd primes
//     up to 43), or, for a prime p whose p-1 is smooth, by Rader's algorithm
//     (a cyclic convolution of length p-1 done with the same Stockham FFT);
//   * with U^a_k = (Z_k + conj Z_{p-k})/2 and U^b_k = (Z_k - conj Z_{p-k})/(2i):
//       y_{2k} = -Im U_k,   y_1 = Re U_0 / 2,   y_{2k+1} = y_{2k-1} + Re U_k,
//     the odd outputs being a prefix sum (one warp per line pair).
// Derivation: substituting t -> p - t shows that the even part
// sin(pi t/p)(x_t + x_{p-t}) contributes only to the cosine sum, where
// 2 sin(pi t/p) cos(2 pi t k/p) = sin(pi t(2k+1)/p) - sin(pi t(2k-1)/p) gives
// Re U_k = y_{2k+1} - y_{2k-1}; the odd part (x_t - x_{p-t})/2 contributes only
// to the sine sum, giving -Im U_k = y_{2k}.  y_{-1} = -y_1 fixes the start.
#pragma once

#include <cuda_runtime.h>

namespace fpg {

enum DstMode { DST_STOCKHAM = 0, DST_RADER = 1, DST_DENSE = 2 };
constexpr int kMaxRadices = 14;

// Plan for one transform length n (tables in the compute precision T).
struct DstPlan {
  int n, p;        // transform length and p = n + 1
  int mode;        // DstMode
  int N;           // Stockham length: p (Stockham) or p - 1 (Rader)
  int nrad;
  int rad[kMaxRadices];
  const void* W;    // N complex: exp(-2 pi i m / N)
  const void* sinp; // p real: sin(pi j / p)
  const void* Bhat; // N complex (Rader): DFT_N of exp(-2 pi i g^{-c}/p), divided by N
  const void* dense;// 2p real: sin(pi m / p) for the dense fallback
  const int* pin;   // N (Rader): g^b mod p
  const int* pout;  // N (Rader): g^{-a} mod p
};

template <typename T>
struct C2 {
  T x, y;
};

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return C2<T>{a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return C2<T>{a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ C2<T> cconj(C2<T> a) { return C2<T>{a.x, -a.y}; }

// Radix-R DFT (forward sign) of v[0..R) with results stored to out[r * os].
// Constants w_R^m = W[m * (N / R)].
template <int R, typename T>
__device__ __forceinline__ void dft_small(C2<T>* v, const C2<T>* __restrict__ W, int N, C2<T>* out, int os) {
  if constexpr (R == 2) {
    out[0] = cadd(v[0], v[1]);
    out[os] = csub(v[0], v[1]);
  } else if constexpr (R == 4) {
    const C2<T> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const C2<T> t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    const C2<T> t3{d.y, -d.x};  // -i (v1 - v3)
    out[0] = cadd(t0, t2);
    out[os] = cadd(t1, t3);
    out[2 * os] = csub(t0, t2);
    out[3 * os] = csub(t1, t3);
  } else {
    // odd R: pair q with R - q.  s_q = v_q + v_{R-q}, d_q = v_q - v_{R-q};
    // X_k = v_0 + sum_q s_q cos(2 pi q k/R) - i sum_q d_q sin(2 pi q k/R).
    constexpr int H = (R - 1) / 2;
    const int step = N / R;
    C2<T> x0 = v[0];
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      const C2<T> a = v[q], b = v[R - q];
      v[q] = cadd(a, b);
      v[R - q] = csub(a, b);
      x0 = cadd(x0, v[q]);
    }
    out[0] = x0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      C2<T> A = v[0], Bs{T(0), T(0)};
#pragma unroll
      for (int q = 1; q <= H; ++q) {
        const int m = (q * k) % R;
        const C2<T> w = W[m * step];  // (cos, -sin)(2 pi m / R)
        A.x = fma(v[q].x, w.x, A.x);
        A.y = fma(v[q].y, w.x, A.y);
        Bs.x = fma(v[R - q].x, -w.y, Bs.x);
        Bs.y = fma(v[R - q].y, -w.y, Bs.y);
      }
      out[k * os] = C2<T>{A.x + Bs.y, A.y - Bs.x};
      out[(R - k) * os] = C2<T>{A.x - Bs.y, A.y + Bs.x};
    }
  }
}

// One Stockham radix-R stage over Q sequences of length N (pitch `pitch`).
template <int R, typename T>
__device__ __forceinline__ void stockham_stage(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, int Q, int N,
                                               int Ns, int pitch, const C2<T>* __restrict__ W) {
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
    dft_small<R, T>(v, W, N, out + q * pitch + (j - jm) * R + jm, Ns);
  }
}

// Power-of-two stages (radices 2, 4, 8, 16) with compile-time register DFTs;
// defined with the register DFTs (fpg_dstline.cuh), used by the MAXR = 16 family.
template <typename T>
__device__ void stockham_pow2(int R, const C2<T>* in, C2<T>* out, int Q, int N, int Ns, int pitch, const C2<T>* W);

// MAXR bounds the radices compiled into one kernel: a kernel built for small
// radices does not carry the register footprint of the large ones.  MAXR = 16
// is the power-of-two family (radices 2, 4, 8, 16 only).
template <typename T, int MAXR>
__device__ __forceinline__ void stockham_dispatch(int R, const C2<T>* in, C2<T>* out, int Q, int N, int Ns,
                                                  int pitch, const C2<T>* W) {
  if constexpr (MAXR == 16) {
    stockham_pow2<T>(R, in, out, Q, N, Ns, pitch, W);
    return;
  }
  switch (R) {
    case 2: stockham_stage<2, T>(in, out, Q, N, Ns, pitch, W); break;
    case 3: stockham_stage<3, T>(in, out, Q, N, Ns, pitch, W); break;
    case 4: stockham_stage<4, T>(in, out, Q, N, Ns, pitch, W); break;
    case 5: stockham_stage<5, T>(in, out, Q, N, Ns, pitch, W); break;
    default:
      if constexpr (MAXR >= 13) {
        switch (R) {
          case 7: stockham_stage<7, T>(in, out, Q, N, Ns, pitch, W); break;
          case 11: stockham_stage<11, T>(in, out, Q, N, Ns, pitch, W); break;
          case 13: stockham_stage<13, T>(in, out, Q, N, Ns, pitch, W); break;
          default:
            if constexpr (MAXR >= 19) {
              switch (R) {
                case 17: stockham_stage<17, T>(in, out, Q, N, Ns, pitch, W); break;
                case 19: stockham_stage<19, T>(in, out, Q, N, Ns, pitch, W); break;
                default:
                  if constexpr (MAXR >= 43) {
                    switch (R) {
                      case 23: stockham_stage<23, T>(in, out, Q, N, Ns, pitch, W); break;
                      case 29: stockham_stage<29, T>(in, out, Q, N, Ns, pitch, W); break;
                      case 31: stockham_stage<31, T>(in, out, Q, N, Ns, pitch, W); break;
                      case 37: stockham_stage<37, T>(in, out, Q, N, Ns, pitch, W); break;
                      case 41: stockham_stage<41, T>(in, out, Q, N, Ns, pitch, W); break;
                      case 43: stockham_stage<43, T>(in, out, Q, N, Ns, pitch, W); break;
                      default: break;  // plans only contain the radices above
                    }
                  }
              }
            }
        }
      }
  }
}

// Radix family a plan needs: 16 for plans of radices 2, 4, 8, 16 with an 8 or a
// 16 among them, else the largest radix rounded up to 5, 13, 19 or 43.
__host__ __device__ inline int plan_maxr(const DstPlan& pl) {
  int mx = 2;
  bool pow2 = true;
  for (int i = 0; i < pl.nrad; ++i) {
    mx = pl.rad[i] > mx ? pl.rad[i] : mx;
    pow2 = pow2 && (pl.rad[i] == 2 || pl.rad[i] == 4 || pl.rad[i] == 8 || pl.rad[i] == 16);
  }
  if (pow2 && mx >= 8) return 16;
  return mx <= 5 ? 5 : (mx <= 13 ? 13 : (mx <= 19 ? 19 : 43));
}

// Runs all stages; returns the buffer holding the result (b0 or b1).
template <typename T, int MAXR>
__device__ __forceinline__ C2<T>* stockham_fft(const DstPlan& pl, C2<T>* b0, C2<T>* b1, int Q, int pitch,
                                               const C2<T>* W) {
  C2<T>* in = b0;
  C2<T>* out = b1;
  int Ns = 1;
  for (int s = 0; s < pl.nrad; ++s) {
    const int R = pl.rad[s];
    stockham_dispatch<T, MAXR>(R, in, out, Q, pl.N, Ns, pitch, W);
    __syncthreads();
    Ns *= R;
    C2<T>* t = in;
    in = out;
    out = t;
  }
  return in;
}

// Shared-memory footprint (bytes) of the engine for Q line pairs.
template <typename T>
__host__ __device__ inline size_t dst_smem_bytes(int p, int N, int Q, int mode) {
  size_t b = 2 * sizeof(C2<T>) * (size_t)Q * p;  // two ping-pong buffers
  b += sizeof(C2<T>) * (size_t)N;                // twiddles
  b += sizeof(T) * (size_t)p;                    // sin(pi j/p)
  if (mode == DST_RADER) b += sizeof(C2<T>) * (size_t)N + 2 * sizeof(int) * (size_t)N + 2 * sizeof(C2<T>) * Q;
  return b + 64;
}

// Pointers into the engine's shared memory.
template <typename T>
struct DstSmem {
  C2<T>* b0;
  C2<T>* b1;
  C2<T>* W;
  T* sinp;
  C2<T>* Bhat;
  int* pin;
  int* pout;
  C2<T>* z0;  // [Q] z_0 of each sequence (Rader)
  C2<T>* zs;  // [Q] sum of each sequence (Rader)
  T* xin;     // real input lines [2Q][n] (aliases b1)
};

template <typename T>
__device__ __forceinline__ DstSmem<T> dst_smem_carve(unsigned char* base, const DstPlan& pl, int Q) {
  DstSmem<T> s;
  C2<T>* c = reinterpret_cast<C2<T>*>(base);
  s.b0 = c;
  s.b1 = c + (size_t)Q * pl.p;
  s.W = s.b1 + (size_t)Q * pl.p;
  C2<T>* after = s.W + pl.N;
  if (pl.mode == DST_RADER) {
    s.Bhat = after;
    s.z0 = s.Bhat + pl.N;
    s.zs = s.z0 + Q;
    after = s.zs + Q;
  } else {
    s.Bhat = s.z0 = s.zs = nullptr;
  }
  s.sinp = reinterpret_cast<T*>(after);
  int* ip = reinterpret_cast<int*>(s.sinp + pl.p);
  if (pl.mode == DST_RADER) {
    s.pin = ip;
    s.pout = ip + pl.N;
  } else {
    s.pin = s.pout = nullptr;
  }
  s.xin = reinterpret_cast<T*>(s.b1);
  return s;
}

// Copy the plan's tables into shared memory (call once per CTA, then sync).
template <typename T>
__device__ __forceinline__ void dst_load_tables(const DstPlan& pl, DstSmem<T>& s) {
  const C2<T>* W = reinterpret_cast<const C2<T>*>(pl.W);
  const T* sp = reinterpret_cast<const T*>(pl.sinp);
  for (int i = threadIdx.x; i < pl.N; i += blockDim.x) s.W[i] = W[i];
  for (int i = threadIdx.x; i < pl.p; i += blockDim.x) s.sinp[i] = sp[i];
  if (pl.mode == DST_RADER) {
    const C2<T>* Bh = reinterpret_cast<const C2<T>*>(pl.Bhat);
    for (int i = threadIdx.x; i < pl.N; i += blockDim.x) {
      s.Bhat[i] = Bh[i];
      s.pin[i] = pl.pin[i];
      s.pout[i] = pl.pout[i];
    }
  }
}

// DST-I of the 2Q real lines s.xin[l * n + t] (lines >= nl must hold zeros).
// Returns a pointer to the outputs y[l * n + k] (staged in shared memory).
// Must be called by the whole CTA; contains __syncthreads().
template <typename T, int MAXR>
__device__ T* dst_lines(const DstPlan& pl, DstSmem<T>& s, int Q) {
  const int n = pl.n, p = pl.p;
  // 1. pack line pairs into z (b0), j = 0..p-1
  for (int idx = threadIdx.x; idx < Q * p; idx += blockDim.x) {
    const int q = idx / p, j = idx - q * p;
    const T* xa = s.xin + (size_t)(2 * q) * n;
    const T* xb = xa + n;
    T a1 = 0, a2 = 0, b1 = 0, b2 = 0;
    if (j >= 1) {  // x_j and x_{p-j}, both inside 1..n
      a1 = xa[j - 1];
      b1 = xb[j - 1];
      a2 = xa[p - j - 1];
      b2 = xb[p - j - 1];
    }
    const T sj = s.sinp[j];
    const T ha = T(0.5) * (a1 - a2), hb = T(0.5) * (b1 - b2);
    s.b0[(size_t)q * p + j] = C2<T>{fma(sj, a1 + a2, ha), fma(sj, b1 + b2, hb)};
  }
  __syncthreads();
  // 2. DFT of length p
  C2<T>* Z;
  C2<T>* freebuf;
  if (pl.mode == DST_STOCKHAM) {
    Z = stockham_fft<T, MAXR>(pl, s.b0, s.b1, Q, p, s.W);
    freebuf = (Z == s.b0) ? s.b1 : s.b0;
  } else {
    const int N = pl.N;
    // keep z_0 and sum_j z_j, gather A_b = z_{g^b} into b1
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = wid; q < Q; q += nw) {
      T sx = 0, sy = 0;
      for (int j = lane; j < p; j += 32) {
        const C2<T> v = s.b0[(size_t)q * p + j];
        sx += v.x;
        sy += v.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0) {
        s.zs[q] = C2<T>{sx, sy};
        s.z0[q] = s.b0[(size_t)q * p];
      }
    }
    for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
      const int q = idx / N, b = idx - q * N;
      s.b1[(size_t)q * p + b] = s.b0[(size_t)q * p + s.pin[b]];
    }
    __syncthreads();
    C2<T>* A = stockham_fft<T, MAXR>(pl, s.b1, s.b0, Q, p, s.W);
    for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
      const int q = idx / N, b = idx - q * N;
      C2<T>& v = A[(size_t)q * p + b];
      v = cconj(cmul(v, s.Bhat[b]));
    }
    __syncthreads();
    C2<T>* other = (A == s.b0) ? s.b1 : s.b0;
    C2<T>* Cv = stockham_fft<T, MAXR>(pl, A, other, Q, p, s.W);
    C2<T>* X = (Cv == s.b0) ? s.b1 : s.b0;
    for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
      const int q = idx / N, a = idx - q * N;
      X[(size_t)q * p + s.pout[a]] = cadd(s.z0[q], cconj(Cv[(size_t)q * p + a]));
    }
    for (int q = threadIdx.x; q < Q; q += blockDim.x) X[(size_t)q * p] = s.zs[q];
    __syncthreads();
    Z = X;
    freebuf = Cv;
  }
  // 3. unpack + prefix sums into the free buffer, viewed as real [2Q][n]
  T* y = reinterpret_cast<T*>(freebuf);
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int K = (p + 1) / 2;  // k = 0..K-1 produce every output y_1..y_n
    const int ck = (K + 31) / 32;
    for (int q = wid; q < Q; q += nw) {
      const C2<T>* Zq = Z + (size_t)q * p;
      T* ya = y + (size_t)(2 * q) * n;
      T* yb = ya + n;
      const int k0 = lane * ck, k1 = min(K, k0 + ck);
      T sa = 0, sb = 0;
      for (int k = k0; k < k1; ++k) {
        const C2<T> zk = Zq[k], zc = cconj(Zq[k == 0 ? 0 : p - k]);
        // Re U^a = (zk.x + zc.x)/2, Re U^b = Im of (Z_k - conj Z_{p-k})/(2i) part: (zk.y - zc.y)/2
        T ra = T(0.5) * (zk.x + zc.x), rb = T(0.5) * (zk.y - zc.y);
        if (k == 0) { ra *= T(0.5); rb *= T(0.5); }
        sa += ra;
        sb += rb;
      }
      // exclusive scan of the lane totals
      T pa = sa, pb = sb;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T ta = __shfl_up_sync(0xffffffffu, pa, o), tb = __shfl_up_sync(0xffffffffu, pb, o);
        if (lane >= o) { pa += ta; pb += tb; }
      }
      T acca = pa - sa, accb = pb - sb;
      for (int k = k0; k < k1; ++k) {
        const C2<T> zk = Zq[k], zc = cconj(Zq[k == 0 ? 0 : p - k]);
        T ra = T(0.5) * (zk.x + zc.x), rb = T(0.5) * (zk.y - zc.y);
        if (k == 0) { ra *= T(0.5); rb *= T(0.5); }
        acca += ra;
        accb += rb;
        if (2 * k + 1 <= n) {
          ya[2 * k] = acca;
          yb[2 * k] = accb;
        }
        if (k >= 1 && 2 * k <= n) {
          // y_{2k} = -Im U_k:  Im U^a = (zk.y + zc.y)/2 ; U^b = (Z_k - conj Z_{p-k})/(2i) -> Im = -(zk.x - zc.x)/2
          ya[2 * k - 1] = -T(0.5) * (zk.y + zc.y);
          yb[2 * k - 1] = T(0.5) * (zk.x - zc.x);
        }
      }
    }
  }
  __syncthreads();
  return y;
}

}  // namespace fpg
