// Integer arithmetic of the tensor-core window sums (fpe_tc.cu), kept apart
// so that the host test (tests/native/tc_arith_host.cu) compiles the same
// code: the balanced base-128 digits of the 69-bit fixed-point operands and
// their bf16 encoding, the join of the ten exact fp32 accumulators (one per
// kept digit-pair diagonal) into one 128-bit integer, and the 64-bit-mantissa
// complex values (xh) in which a work item's blocks are combined by Horner's
// scheme.
#pragma once

#include <cstdint>
#include <cstring>

#include "fpe_device.cuh"

namespace fpe {

constexpr int kTB = 32;   // terms per block
constexpr int kSl = 10;   // 7-bit digits per operand (slices)
constexpr int kAcc = 10;  // kept digit-pair diagonals t = s + s' <= 9, one fp32 accumulator each

__host__ __device__ __forceinline__ uint32_t tc_fbits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

__host__ __device__ __forceinline__ float tc_bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}

__host__ __device__ __forceinline__ int tc_clz64(unsigned long long m) {
#ifdef __CUDA_ARCH__
  return __clzll(m);
#else
  return m ? __builtin_clzll(m) : 64;
#endif
}

// ---------------------------------------------------------------------------
// A complex value with 64-bit mantissas, ((-1)^sx x + i (-1)^sy y) 2^(e - 63),
// max(x, y) in [2^63, 2^64) or both 0: the per-block Horner inside a work
// item runs in it.  A product or a sum is within 2^-60 of the exact value
// relative to its operands (two truncated high products or aligned
// operands, each halved); a thread's chain of such steps is at most 64 long
// (it is folded into 128 bits after that), which keeps its error below
// 2^-54 of its terms' sum.
// ---------------------------------------------------------------------------
struct xh {
  unsigned long long x, y;
  int sx, sy;
  long long e;
};

__host__ __device__ __forceinline__ xh xh_norm(unsigned long long x, int sx, unsigned long long y, int sy,
                                               long long e) {
  const unsigned long long m = x | y;  // the same leading bit as max(x, y)
  xh r;
  if (m == 0) {
    r.x = r.y = 0;
    r.sx = r.sy = 0;
    r.e = 0;
    return r;
  }
  const int sh = tc_clz64(m);
  r.x = x << sh;
  r.y = y << sh;
  r.sx = r.x ? sx : 0;
  r.sy = r.y ? sy : 0;
  r.e = e - sh;
  return r;
}

// top 64 bits of a 128-bit magnitude pair (value X 2^(e - 126) as in xint)
__host__ __device__ __forceinline__ xh xh_from128(u128 X, int sx, u128 Y, int sy, long long e) {
  const u128 m = X | Y;  // the same leading bit as max(X, Y)
  if (m == 0) return xh_norm(0, 0, 0, 0, 0);
  const int sh = clz128(m);  // bring the top bit to 127: the larger top half is then normalised
  X <<= sh;
  Y <<= sh;
  xh r;
  r.x = (unsigned long long)(X >> 64);
  r.y = (unsigned long long)(Y >> 64);
  r.sx = r.x ? sx : 0;
  r.sy = r.y ? sy : 0;
  r.e = e - sh + 1;
  return r;
}

__host__ __device__ __forceinline__ xh xh_from_xint(const xint &v) { return xh_from128(v.x, v.sx, v.y, v.sy, v.e); }

__host__ __device__ __forceinline__ xint xint_from_xh(const xh &v) {
  return xint_norm((u128)v.x << 62, v.sx, (u128)v.y << 62, v.sy, v.e + 1);
}

// signed-magnitude a + b (halved, so no overflow)
__host__ __device__ __forceinline__ void sadd64h(unsigned long long a, int sa, unsigned long long b, int sb,
                                                 unsigned long long &r, int &sr) {
  a >>= 1;
  b >>= 1;
  if (sa == sb) {
    r = a + b;
    sr = sa;
  } else if (a >= b) {
    r = a - b;
    sr = sa;
  } else {
    r = b - a;
    sr = sb;
  }
}

__host__ __device__ __forceinline__ xh xh_mul(const xh &a, const xh &b) {
  const unsigned long long p1 = umulhi64(a.x, b.x), p2 = umulhi64(a.y, b.y);
  const unsigned long long p3 = umulhi64(a.x, b.y), p4 = umulhi64(a.y, b.x);
  unsigned long long re, im;
  int sre, sim;
  sadd64h(p1, a.sx ^ b.sx, p2, 1 ^ a.sy ^ b.sy, re, sre);
  sadd64h(p3, a.sx ^ b.sy, p4, a.sy ^ b.sx, im, sim);
  // p = a b 2^-64 in units of 2^(ea + eb - 126), halved: exponent ea + eb - 126 + 64 + 1 + 63
  return xh_norm(re, sre, im, sim, a.e + b.e + 2);
}

__host__ __device__ __forceinline__ xh xh_add(const xh &a, const xh &b) {
  if (!a.x && !a.y) return b;
  if (!b.x && !b.y) return a;
  const xh &hi = a.e >= b.e ? a : b, &lo = a.e >= b.e ? b : a;
  const long long d = hi.e - lo.e;
  const unsigned long long lx = d < 64 ? (lo.x >> d) : 0ull, ly = d < 64 ? (lo.y >> d) : 0ull;
  unsigned long long rx, ry;
  int sx, sy;
  sadd64h(hi.x, hi.sx, lx, lo.sx, rx, sx);
  sadd64h(hi.y, hi.sy, ly, lo.sy, ry, sy);
  return xh_norm(rx, rx ? sx : 0, ry, ry ? sy : 0, hi.e + 1);
}

// ---------------------------------------------------------------------------
// Digits.  Balanced base-128 digits of F < 2^69: F = sum_j d_j 128^(9 - j)
// with d_j in [-64, 63] for j > 0 and d_0 in [0, 64].  Adding
// B = sum_j 64 128^j makes them plain chunks c_j = d_j + 64 of G = F + B
// (7 bits each; the top one, everything above bit 63, at most 128).  Each
// chunk is returned as the bits of the float 2^23 + c_j, from which one
// fused multiply-add by +-1 gives +-d_j exactly (bf16_pair).  Products of
// two digits stay within 2^12, and the ten slice pairs of one accumulator
// over a 64-long dot product within 10 x 2^18 < 2^22: fp32 accumulation is
// exact with room to spare.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void bchunks70(u128 F, uint32_t (&x)[kSl]) {
  const u128 G = F + (((u128)0x20 << 64) | 0x4081020408102040ull);
  const unsigned long long lo = (unsigned long long)G, hi = (unsigned long long)(G >> 64);
  x[0] = 0x4B000000u | (uint32_t)((hi << 1) | (lo >> 63));
#pragma unroll
  for (int j = 1; j < kSl; ++j) x[j] = 0x4B000000u | ((uint32_t)(lo >> (7 * (kSl - 1 - j))) & 127u);
}

// the multiplier and addend that turn a chunk's float 2^23 + c into
// (-1)^neg (c - 64), exactly
struct DigitSign {
  float s, k;
};
__host__ __device__ __forceinline__ DigitSign digit_sign(uint32_t neg) {
  DigitSign r;
  r.s = neg ? -1.0f : 1.0f;
  r.k = neg ? 8388672.0f : -8388672.0f;
  return r;
}

// two signed digits as a pair of bf16 (a in the low half, i.e. at the lower
// address): the digits are small integers, exact in bf16, so the bf16 is the
// float's upper half
__host__ __device__ __forceinline__ uint32_t bf16_pair(uint32_t xa, DigitSign sa, uint32_t xb, DigitSign sb) {
  const uint32_t a = tc_fbits(fmaf(tc_bitsf(xa), sa.s, sa.k));
  const uint32_t b = tc_fbits(fmaf(tc_bitsf(xb), sb.s, sb.k));
#ifdef __CUDA_ARCH__
  return __byte_perm(a, b, 0x7632);
#else
  return (a >> 16) | (b & 0xffff0000u);
#endif
}

// X 2^-sr (sr may be negative), saturated below 2^70
__host__ __device__ __forceinline__ u128 shift_to70(u128 X, int sr) {
  const u128 cap = ((u128)1 << 70) - 1;
  if (sr >= 128) return 0;
  if (sr >= 0) {
    const u128 F = X >> sr;
    return F > cap ? cap : F;
  }
  if (sr <= -70 || (X >> (70 + sr)) != 0) return cap;
  return X << (-sr);
}

// X = sum_t v_t 128^(9 - t) over the ten accumulators v_t of one output (t =
// the digit-pair diagonal), as a 128-bit magnitude and a sign.  Each v_t is
// an integer below 2^22 in magnitude held exactly in fp32; adding 1.5 2^23
// puts it in the low mantissa bits, so the float's bits are
// w_t = v_t + 0x4B400000.  The pairs v_2j 128 + v_2j+1 (below 2^29.1) come
// from the w's in wrap-around 32-bit arithmetic, and three 32 x 32 + 64-bit
// products join them.
__host__ __device__ __forceinline__ void join_vals(const float (&v)[kAcc], u128 &mag, int &neg) {
  int pr[kAcc / 2];
#pragma unroll
  for (int j = 0; j < kAcc / 2; ++j) {
    const uint32_t wa = tc_fbits(v[2 * j] + 12582912.0f);
    const uint32_t wb = tc_fbits(v[2 * j + 1] + 12582912.0f);
    pr[j] = (int)(wa * 128u + wb - 129u * 0x4B400000u);
  }
  const long long lo = (long long)pr[2] * (1ll << 28) + (long long)pr[3] * (1ll << 14) + pr[4];
  const long long hi = (long long)pr[0] * (1ll << 14) + pr[1];
  const __int128 X = ((__int128)hi << 42) + (__int128)lo;
  neg = X < 0;
  mag = (u128)(neg ? -X : X);
}

}  // namespace fpe
