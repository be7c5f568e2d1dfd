// Exact, order-independent sums of doubles across a warp, a CTA and a thread-block
// cluster, for the projections h_{i,j} = (w, v_i) of the Arnoldi step (Alg. 2's
// modified Gram-Schmidt) and the norm that closes it.
//
// Each double p = (-1)^s m 2^(e - 1075) (m < 2^53, e the biased exponent field, 1 for
// subnormals) is written as a fixed-point integer a = m 2^10 / 2^(E - e) relative to
// the largest exponent E among the values summed together (low bits beyond 2^(E - 1085)
// are dropped: at most 2^-62 of the largest term each).  Integers are summed exactly
// as 20-bit chunks with the integer warp reductions (redux.sync), so the result does
// not depend on the order of the terms within a warp, of the warps within a CTA or of
// the CTAs within a cluster: every CTA of a cluster obtains the same bits.  (Another
// launch shape groups the terms into other warps, so the dropped low bits, and rarely
// the last bit of the result, may differ.)  The one rounding is the final conversion
// of the summed integer to double (round to nearest even).  The error against the exact sum of the inputs is at most
// (number of terms) 2^-62 of the largest term plus that rounding, below the error of a
// floating-point summation tree of the same terms.
//
// These sums run on the integer pipes.  On this GPU the FP64 pipe retires a warp
// instruction in about 16 SM cycles whether one lane or all 32 are active, so a
// floating-point tree spends about as much FP64 time on the reduction of one
// projection as 9 elements of the dot product do per thread.
//
// Tuples: value = (c3 2^60 + c2 2^40 + c1 2^20 + c0) 2^(E - 1085), with c0, c1, c2 sums of
// 20-bit chunks and c3 a signed sum; packed in an int4 as {c0, c1, c2, c3 * 2048 + E}
// (E < 2048; |c3| < 2^16 for up to 16 x 16 x 32 terms, chunk sums c0..c2 < 2^25).
#pragma once

#include <cuda_runtime.h>

namespace fpg {
namespace xs {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ __int128 join(int c0, int c1, int c2, int c3) {
  return ((__int128)c3 << 60) + ((__int128)c2 << 40) + ((__int128)c1 << 20) + (__int128)c0;
}

__device__ __forceinline__ int4 pack(unsigned E, int c0, int c1, int c2, int c3) {
  return make_int4(c0, c1, c2, c3 * 2048 + (int)E);
}
__device__ __forceinline__ unsigned tuple_exp(int4 t) { return (unsigned)(t.w & 2047); }
__device__ __forceinline__ int tuple_top(int4 t) { return t.w >> 11; }

// Sum over the 32 lanes of a warp (all lanes must call; each passes its own term).
__device__ __forceinline__ int4 warp_sum_exact(double p) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(p);
  const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned eff = e ? e : 1u;
  const unsigned E = __reduce_max_sync(kFull, eff);
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull));
  const unsigned d = E - eff;
  long long a = d < 63u ? ((m << 10) >> d) : 0ll;  // m 2^10 < 2^63
  if (b >> 63) a = -a;
  const int c0 = __reduce_add_sync(kFull, (int)(a & 0xFFFFF));
  const int c1 = __reduce_add_sync(kFull, (int)((a >> 20) & 0xFFFFF));
  const int c2 = __reduce_add_sync(kFull, (int)((a >> 40) & 0xFFFFF));
  const int c3 = __reduce_add_sync(kFull, (int)(a >> 60));
  return pack(E, c0, c1, c2, c3);
}

// Sum of tuples held one per lane (lanes without a tuple pass valid = false); the
// result is returned to every lane.
__device__ __forceinline__ int4 warp_sum_tuples(int4 t, bool valid) {
  const unsigned e = valid ? tuple_exp(t) : 0u;
  const unsigned E = __reduce_max_sync(kFull, e);
  __int128 v = valid ? join(t.x, t.y, t.z, tuple_top(t)) : (__int128)0;
  const unsigned d = E - e;
  v = d < 100u ? (v >> d) : (__int128)0;
  const int c0 = __reduce_add_sync(kFull, (int)(v & 0xFFFFF));
  const int c1 = __reduce_add_sync(kFull, (int)((v >> 20) & 0xFFFFF));
  const int c2 = __reduce_add_sync(kFull, (int)((v >> 40) & 0xFFFFF));
  const int c3 = __reduce_add_sync(kFull, (int)(v >> 60));
  return pack(E, c0, c1, c2, c3);
}

// The tuple's value as the nearest double (ties to even); NaN when a term was not finite.
__device__ __forceinline__ double tuple_to_double(int4 t) {
  const unsigned E = tuple_exp(t);
  if (E >= 2047u) return __longlong_as_double(0x7FF8000000000000ll);
  const __int128 v = join(t.x, t.y, t.z, tuple_top(t));
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
  unsigned long long top = lo;
  int sh = 0;
  if (hi) {
    // keep the leading 64 bits; the bits shifted out only decide ties (sticky bit)
    sh = 64 - __clzll((long long)hi);
    top = (unsigned long long)(u >> sh);
    const unsigned long long out = sh >= 64 ? lo : (lo & ((1ull << sh) - 1ull));
    top |= out ? 1ull : 0ull;
  }
  const double r = ldexp(__ull2double_rn(top), sh + (int)E - 1085);
  return neg ? -r : r;
}

// ---- cluster exchange: every CTA pushes its tuple into slot [rank] of every CTA with
// st.async, completing on that CTA's mbarrier (16 bytes per CTA of the cluster).

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned cluster_addr(unsigned local, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_init_cluster(unsigned long long* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The one local arrival of a phase, announcing `bytes` still to come.
__device__ __forceinline__ void mbar_expect(unsigned long long* mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// Wait for phase `parity` with cluster-scope acquire (the bytes come from other
// CTAs); false after `limit` unsuccessful tries.
__device__ __forceinline__ bool mbar_wait_cluster(unsigned long long* mbar, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void st_async_tuple(unsigned remote, int4 v, unsigned remote_mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   remote),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(remote_mbar)
               : "memory");
}

// Split cluster barrier (every thread of every CTA of the cluster).
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

}  // namespace xs
}  // namespace fpg
