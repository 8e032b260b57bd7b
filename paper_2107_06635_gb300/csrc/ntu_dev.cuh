// Device-side numerics shared by the NTU kernels: complex helpers, CTA
// reductions and the small dense linear-algebra routines of the bond update
// (one-sided Jacobi SVD, Householder QR / Hermitian tridiagonalisation,
// implicit symmetric tridiagonal QR).  All CTA routines assume
// blockDim.x == NTU_CTA threads.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "df_bits.cuh"

#define NTU_CTA 256
#define NTU_WARPS (NTU_CTA / 32)

namespace ntu {

// ------------------------------------------------------------------ complex
__device__ __forceinline__ double2 cz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// a * b + c
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}
// conj(a) * b + c
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
// c - a * b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
  c.x = fma(-a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
// c - a * conj(b)
__device__ __forceinline__ double2 cfmsc(double2 a, double2 b, double2 c) {
  c.x = fma(-a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// x = hi + lo with hi = bf16(x) and lo = bf16(x - hi): the split operands of
// the three-pass tensor-core products.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Store complex value (re, im) of complex row r, complex column kc into a
// split [hi | lo] BF16 operand with row pitch `pitch` and lo offset `krp`.
// doubled = 0: interleaved (re, im) row (a B operand).  doubled = 1: the
// real rows (r/64)*128 + r%64 and +64 receive (re, -im) and (im, re) (a
// doubled A operand: one real GEMM then yields Re in the first 64 and Im in
// the last 64 rows of each 128-row tile).
__device__ __forceinline__ void store_split(__nv_bfloat16* base, long long r, long long kc,
                                            int pitch, int krp, float re, float im,
                                            int doubled) {
  // pitch and krp are even, so every (re, im) pair is a 4-byte aligned word
  __nv_bfloat16 h0, l0, h1, l1;
  split_bf16(re, h0, l0);
  split_bf16(im, h1, l1);
  if (!doubled) {
    __nv_bfloat162* p = reinterpret_cast<__nv_bfloat162*>(base + r * pitch + 2 * kc);
    p[0] = __halves2bfloat162(h0, h1);
    p[krp / 2] = __halves2bfloat162(l0, l1);
  } else {
    // -im splits into (-hi, -lo) exactly
    __nv_bfloat162* pr =
        reinterpret_cast<__nv_bfloat162*>(base + ((r / 64) * 128 + (r % 64)) * pitch + 2 * kc);
    __nv_bfloat162* pi = pr + 32LL * pitch;
    pr[0] = __halves2bfloat162(h0, __hneg(h1));
    pr[krp / 2] = __halves2bfloat162(l0, __hneg(l1));
    pi[0] = __halves2bfloat162(h1, h0);
    pi[krp / 2] = __halves2bfloat162(l1, l0);
  }
}
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  __nv_bfloat162 t = __halves2bfloat162(a, b);
  return *reinterpret_cast<uint32_t*>(&t);
}
// Four consecutive complex columns kc .. kc+3 (kc a multiple of 4) of complex
// row r in the layout of store_split: the hi halves go out as one 16-byte
// store and the lo halves as another (two each for a doubled operand).
__device__ __forceinline__ void store_split4(__nv_bfloat16* base, long long r, long long kc,
                                             int pitch, int krp, float4 re, float4 im,
                                             int doubled) {
  const float rv[4] = {re.x, re.y, re.z, re.w}, iv[4] = {im.x, im.y, im.z, im.w};
  __nv_bfloat16 rh[4], rl[4], ih[4], il[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) { split_bf16(rv[q], rh[q], rl[q]); split_bf16(iv[q], ih[q], il[q]); }
  if (!doubled) {
    __nv_bfloat16* p = base + r * pitch + 2 * kc;
    *reinterpret_cast<uint4*>(p) = make_uint4(pack_bf16(rh[0], ih[0]), pack_bf16(rh[1], ih[1]),
                                              pack_bf16(rh[2], ih[2]), pack_bf16(rh[3], ih[3]));
    *reinterpret_cast<uint4*>(p + krp) = make_uint4(pack_bf16(rl[0], il[0]), pack_bf16(rl[1], il[1]),
                                                    pack_bf16(rl[2], il[2]), pack_bf16(rl[3], il[3]));
  } else {
    __nv_bfloat16* pr = base + ((r / 64) * 128 + (r % 64)) * pitch + 2 * kc;
    __nv_bfloat16* pi = pr + 64LL * pitch;
    *reinterpret_cast<uint4*>(pr) =
        make_uint4(pack_bf16(rh[0], __hneg(ih[0])), pack_bf16(rh[1], __hneg(ih[1])),
                   pack_bf16(rh[2], __hneg(ih[2])), pack_bf16(rh[3], __hneg(ih[3])));
    *reinterpret_cast<uint4*>(pr + krp) =
        make_uint4(pack_bf16(rl[0], __hneg(il[0])), pack_bf16(rl[1], __hneg(il[1])),
                   pack_bf16(rl[2], __hneg(il[2])), pack_bf16(rl[3], __hneg(il[3])));
    *reinterpret_cast<uint4*>(pi) = make_uint4(pack_bf16(ih[0], rh[0]), pack_bf16(ih[1], rh[1]),
                                               pack_bf16(ih[2], rh[2]), pack_bf16(ih[3], rh[3]));
    *reinterpret_cast<uint4*>(pi + krp) =
        make_uint4(pack_bf16(il[0], rl[0]), pack_bf16(il[1], rl[1]), pack_bf16(il[2], rl[2]),
                   pack_bf16(il[3], rl[3]));
  }
}
// Doubled A operand with planar K: complex column kc of a real row pair
// puts its real-part factor at K position kc and its imaginary-part factor at
// krp/2 + kc (the B operand then holds Re at kc and Im at krp/2 + kc).  The
// row pair receives (re, -im) and (im, re) as in store_split.
__device__ __forceinline__ void store_split_planar(__nv_bfloat16* base, long long r, long long kc,
                                                   int pitch, int krp, float re, float im) {
  __nv_bfloat16 h0, l0, h1, l1;
  split_bf16(re, h0, l0);
  split_bf16(im, h1, l1);
  __nv_bfloat16* pr = base + ((r / 64) * 128 + (r % 64)) * pitch + kc;
  __nv_bfloat16* pi = pr + 64LL * pitch;
  const int half = krp / 2;
  pr[0] = h0; pr[half] = __hneg(h1); pr[krp] = l0; pr[krp + half] = __hneg(l1);
  pi[0] = h1; pi[half] = h0; pi[krp] = l1; pi[krp + half] = l0;
}

__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
// a / b by Smith's method (no squares of b, so no underflow or overflow for
// tiny or huge b).
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  double r = b.x / b.y, den = b.y + b.x * r;
  return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}

// --------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the CTA; every thread gets the result.  sbuf: >= NTU_WARPS*2 doubles.
__device__ __forceinline__ double block_sum(double v, double* sbuf) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sbuf[w] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < NTU_WARPS; ++i) t += sbuf[i];
  return t;
}
__device__ __forceinline__ double2 block_sum2(double2 v, double* sbuf) {
  v = warp_sum2(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sbuf[2 * w] = v.x; sbuf[2 * w + 1] = v.y; }
  __syncthreads();
  double2 t = cz();
#pragma unroll
  for (int i = 0; i < NTU_WARPS; ++i) { t.x += sbuf[2 * i]; t.y += sbuf[2 * i + 1]; }
  return t;
}
__device__ __forceinline__ double block_min(double v, double* sbuf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sbuf[w] = v;
  __syncthreads();
  double t = sbuf[0];
#pragma unroll
  for (int i = 1; i < NTU_WARPS; ++i) t = fmin(t, sbuf[i]);
  return t;
}
__device__ __forceinline__ double block_max(double v, double* sbuf) {
  v = warp_max(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sbuf[w] = v;
  __syncthreads();
  double t = sbuf[0];
#pragma unroll
  for (int i = 1; i < NTU_WARPS; ++i) t = fmax(t, sbuf[i]);
  return t;
}

// Error codes a kernel may raise through the status word (same values as
// ntu_status in include/ntu.h).
enum { ST_NUMERIC = 4, ST_TIMEOUT = 5 };
// Reason bits recorded next to the status word (status[1]).
enum {
  WHY_SVD_NONFINITE = 1, WHY_ALS_QR = 2, WHY_ALS_NONFINITE = 4, WHY_REPAIR_QR = 8,
  WHY_REPAIR_TRACE = 16, WHY_TC_WAIT = 32, WHY_ALS_SYNC = 64
};
__device__ __forceinline__ void raise_status(int* status, int code, int why = 0) {
  if (status) {
    atomicMax(status, code);
    if (why) atomicOr(status + 1, why);
  }
}

// ------------------------------------------------- Householder reflectors
// Reflector H = I - tau v v^H with v = [1; x/(alpha - beta)] such that
// H^H [alpha; x] = [beta; 0] and beta real, beta = -sign(Re alpha) ||[alpha; x]||
// (the convention of the standard complex Householder QR).  Given alpha and
// ||x||^2, returns tau, beta and the factor that scales x into v.
struct Reflector { double2 tau; double beta; double2 scale; };

// CTA-wide reflector of the vector v[0..len) = [alpha; x].  The norm is taken
// of the vector divided by its largest component, so that entries far below
// the square root of the smallest normal number neither vanish from nor
// zero out the norm.  Reads v only; every thread returns the same result.
__device__ inline Reflector cta_reflector(const double2* v, int len, double* sred) {
  const int tid = threadIdx.x;
  double mx = 0.0;
  for (int i = 1 + tid; i < len; i += NTU_CTA) mx = fmax(mx, fmax(fabs(v[i].x), fabs(v[i].y)));
  mx = block_max(mx, sred);
  const double2 alpha = v[0];
  const double amax = fmax(mx, fmax(fabs(alpha.x), fabs(alpha.y)));
  double xs2 = 0.0;
  if (mx > 0.0) {
    const double inv = 1.0 / amax;
    for (int i = 1 + tid; i < len; i += NTU_CTA) xs2 += cabs2(cscale(v[i], inv));
  }
  xs2 = block_sum(xs2, sred);
  Reflector r;
  if (mx == 0.0 && alpha.y == 0.0) {
    r.tau = cz(); r.beta = alpha.x; r.scale = make_double2(1.0, 0.0);
    return r;
  }
  const double nrm = amax * sqrt(cabs2(cscale(alpha, 1.0 / amax)) + xs2);
  const double beta = alpha.x >= 0.0 ? -nrm : nrm;
  r.beta = beta;
  r.tau = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
  r.scale = cdiv(make_double2(1.0, 0.0), make_double2(alpha.x - beta, alpha.y));
  return r;
}

// ------------------------------------------- double-FP32 arithmetic
// A real number x is carried as an unevaluated sum hi + lo of two FP32
// values (hi = fl32(x), lo = fl32(x - hi)), good to about 2^-48 relative; a
// complex number as float4 (re_hi, im_hi, re_lo, im_lo).  Products use the
// exact FMA residual of hi * hi plus the two cross terms (lo * lo is below
// the format's precision); sums keep the rounding error of the high part
// exactly (two-sum) and add all low-order terms in FP32.  The explicitly
// rounded intrinsics keep the compiler from contracting the error terms.
// On this GPU FP32 issues at 64x the FP64 rate, so the ~12 FP32 operations
// of a real multiply-add cost less than a sixth of one FP64 FMA.
__device__ __forceinline__ float4 df_split(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, ih, __double2float_rn(v.x - (double)rh),
                     __double2float_rn(v.y - (double)ih));
}
__device__ __forceinline__ double2 df_join(float4 a) {
  return make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
}
// The same split from the bit patterns (df_bits.cuh): the same bits, issued
// on the integer and FP32 pipes instead of the conversion and FP64 ones.
// It pays where those limit a kernel (a streaming pass over g) and costs
// where the FP32 pipe does (the double-FP32 products).
__device__ __forceinline__ float4 df_split_bits(double2 v) {
  float rh, rl, ih, il;
  df_split_real(v.x, rh, rl);
  df_split_real(v.y, ih, il);
  return make_float4(rh, ih, rl, il);
}
// (sh, sl) += (xh + xl) (yh + yl)
__device__ __forceinline__ void df_mac1(float& sh, float& sl, float xh, float xl, float yh,
                                        float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  const float t = __fadd_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}
// acc += a * b, or conj(a) * b with CONJ
template <bool CONJ>
__device__ __forceinline__ void df_cmac(float4& acc, float4 a, float4 b) {
  const float s = CONJ ? -1.0f : 1.0f;
  df_mac1(acc.x, acc.z, a.x, a.z, b.x, b.z);                  // re += ar br
  df_mac1(acc.x, acc.z, -s * a.y, -s * a.w, b.y, b.w);        // re -+= ai bi
  df_mac1(acc.y, acc.w, a.x, a.z, b.y, b.w);                  // im += ar bi
  df_mac1(acc.y, acc.w, s * a.y, s * a.w, b.x, b.z);          // im +-= ai br
}

// (sh, sl) += (bh + bl)
__device__ __forceinline__ void df_add1(float& sh, float& sl, float bh, float bl) {
  const float t = __fadd_rn(sh, bh);
  const float z = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(bh, z));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, bl));
}
// Sum of a double-FP32 complex value over the 32 lanes of a warp (all lanes
// receive it).
__device__ __forceinline__ float4 df_warp_sum(float4 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float4 w = make_float4(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o),
                                 __shfl_xor_sync(0xffffffffu, v.z, o), __shfl_xor_sync(0xffffffffu, v.w, o));
    df_add1(v.x, v.z, w.x, w.z);
    df_add1(v.y, v.w, w.y, w.w);
  }
  return v;
}

// -------------------------------------------------- one-sided Jacobi SVD
// SVD of an m x n complex matrix (m, n <= 32) held column-major in shared
// memory with leading dimension 32: A V = U diag(s).  On exit A's first n
// columns hold the left singular vectors U (m x n) sorted by descending
// singular value, s the values, V (n x n) the right singular vectors.  With
// phase != 0 each column pair carries the convention "first entry of u within
// 1e-10 of the largest modulus is real positive".  Columns with zero singular
// value are returned as zero vectors.  For m < n the trailing n - m values
// are zero.  Work space: W (32 x 32 complex) and sw (>= 3*32 doubles + 32
// ints).
struct SvdSmem {
  double2 A[32 * 32];
  double2 V[32 * 32];
  double2 W[32 * 32];
  double s[32];
  double red[2 * NTU_WARPS];
  int perm[32];
  int rotated;
  int bad;        // set when a singular value came out non-finite
};

// Phase convention of an SVD held as S.A = U (m x n columns), S.V = V:
// the first entry of each column of U within 1e-10 of the column's largest
// modulus becomes real positive, V's column taking the same phase (so U S
// V^H is unchanged); one 16-lane group per column.
__device__ inline void cta_svd_phase(SvdSmem& S, int m, int n) {
  const int tid = threadIdx.x, grp = tid >> 4, lane = tid & 15;
  const unsigned mask = 0xffffu << (tid & 16);
  for (int k = grp; k < n; k += 16) {
    double mx = 0.0;
    for (int r = lane; r < m; r += 16) mx = fmax(mx, cabs2(S.A[k * 32 + r]));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(mask, mx, o));
    mx = sqrt(mx);
    int piv = 1 << 30;
    for (int r = lane; r < m; r += 16)
      if (mx > 0.0 && sqrt(cabs2(S.A[k * 32 + r])) >= (1.0 - 1e-10) * mx) piv = min(piv, r);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) piv = min(piv, __shfl_xor_sync(mask, piv, o));
    if (mx > 0.0 && isfinite(mx) && piv < m) {
      double2 up = S.A[k * 32 + piv];
      double a = sqrt(cabs2(up));
      double2 ph = make_double2(up.x / a, -up.y / a);
      for (int r = lane; r < m; r += 16) S.A[k * 32 + r] = cmul(S.A[k * 32 + r], ph);
      for (int r = lane; r < n; r += 16) S.V[k * 32 + r] = cmul(S.V[k * 32 + r], ph);
    }
  }
  __syncthreads();
}

__device__ inline void cta_svd_cols(SvdSmem& S, int m, int n, int phase) {
  const int tid = threadIdx.x;
  const int np = (n + 1) & ~1;          // even number of columns (virtual zero col)
  // V = identity
  for (int i = tid; i < 32 * 32; i += NTU_CTA) {
    int r = i & 31, c = i >> 5;
    S.V[i] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    if (c >= n || r >= m) S.A[i] = cz();
  }
  __syncthreads();
  const int grp = tid >> 4;             // 16 groups of 16 lanes
  const int lane = tid & 15;
  const unsigned mask = 0xffffu << ((tid & 16));
  const double tol = fmax(1e-15, 2.3e-16 * m);
  const double tol2 = tol * tol;
  // Frobenius norm^2 of the input: pairs whose inner product is below
  // 1e-30 of it belong to the numerical null space and are not rotated
  // (their rounding-level inner products would otherwise never converge).
  double fro = 0.0;
  for (int i = tid; i < 32 * 32; i += NTU_CTA) fro += cabs2(S.A[i]);
  fro = block_sum(fro, S.red);
  const double gnull = 1e-30 * fro;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) S.rotated = 0;
    __syncthreads();
    for (int t = 0; t < np - 1; ++t) {
      if (grp < np / 2) {
        int p, q;
        if (grp == 0) { p = t; q = np - 1; }
        else { p = (t + grp) % (np - 1); q = (t - grp + (np - 1)) % (np - 1); }
        if (p > q) { int tmp = p; p = q; q = tmp; }
        if (q < n) {
          double al = 0.0, be = 0.0; double2 ga = cz();
          for (int r = lane; r < m; r += 16) {
            double2 ap = S.A[p * 32 + r], aq = S.A[q * 32 + r];
            al += cabs2(ap); be += cabs2(aq); ga = cfmac(ap, aq, ga);
          }
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) {
            al += __shfl_xor_sync(mask, al, o);
            be += __shfl_xor_sync(mask, be, o);
            ga.x += __shfl_xor_sync(mask, ga.x, o);
            ga.y += __shfl_xor_sync(mask, ga.y, o);
          }
          const double g2 = cabs2(ga);
          const double rg = g2 > 0.0 ? rsqrt(g2) : 0.0;      // 1 / |<a_p, a_q>|
          if (g2 * rg > gnull && g2 > tol2 * (al * be)) {
            // rotate (p, q) so that the pair becomes orthogonal: with
            // zeta = (|a_q|^2 - |a_p|^2) / (2 |g|), t = sign(zeta) /
            // (|zeta| + sqrt(1 + zeta^2)) is the smaller root of
            // t^2 + 2 zeta t - 1 = 0, c = 1 / sqrt(1 + t^2), s = c t
            const double zeta = (be - al) * (0.5 * rg);
            const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = rsqrt(1.0 + tt * tt), s = c * tt;
            const double2 ph = make_double2(ga.x * rg, -ga.y * rg);     // e^{-i phi}
            for (int r = lane; r < m; r += 16) {
              double2 ap = S.A[p * 32 + r], aq = cmul(S.A[q * 32 + r], ph);
              S.A[p * 32 + r] = make_double2(c * ap.x - s * aq.x, c * ap.y - s * aq.y);
              S.A[q * 32 + r] = make_double2(s * ap.x + c * aq.x, s * ap.y + c * aq.y);
            }
            for (int r = lane; r < n; r += 16) {
              double2 vp = S.V[p * 32 + r], vq = cmul(S.V[q * 32 + r], ph);
              S.V[p * 32 + r] = make_double2(c * vp.x - s * vq.x, c * vp.y - s * vq.y);
              S.V[q * 32 + r] = make_double2(s * vp.x + c * vq.x, s * vp.y + c * vq.y);
            }
            if (lane == 0) S.rotated = 1;
          }
        }
      }
      __syncthreads();
    }
    if (!S.rotated) break;
    __syncthreads();
  }
  // singular values = column norms
  for (int c = grp; c < n; c += 16) {
    double a = 0.0;
    for (int r = lane; r < m; r += 16) a += cabs2(S.A[c * 32 + r]);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(mask, a, o);
    if (lane == 0) S.s[c] = sqrt(a);
  }
  __syncthreads();
  if (tid < 32) S.perm[tid] = tid;
  if (tid == 0) {
    int bad = 0;
    for (int j = 0; j < n; ++j) bad |= !isfinite(S.s[j]);
    S.bad = bad;
  }
  __syncthreads();
  if (tid < n) {          // rank of column tid in descending order: a strict total
    // order in which non-finite values rank last, so perm is a permutation
    double sv = S.s[tid];
    if (!isfinite(sv)) sv = -1.0;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double sj = S.s[j];
      if (!isfinite(sj)) sj = -1.0;
      rank += (sj > sv) || (sj == sv && j < tid);
    }
    S.perm[rank] = tid;
  }
  __syncthreads();
  // gather the normalised, sorted columns (U) into W
  for (int i = tid; i < 32 * 32; i += NTU_CTA) {
    int r = i & 31, k = i >> 5;
    double2 u = cz();
    if (k < n && r < m) {
      int src = S.perm[k] & 31;
      double sv = S.s[src];
      if (sv > 0.0 && isfinite(sv)) u = cscale(S.A[src * 32 + r], 1.0 / sv);
    }
    S.W[i] = u;
  }
  __syncthreads();
  // sorted V into A's storage, then V <- A and A <- W
  for (int i = tid; i < 32 * 32; i += NTU_CTA) {
    int r = i & 31, k = i >> 5;
    S.A[i] = (k < n && r < n) ? S.V[(S.perm[k] & 31) * 32 + r] : cz();
  }
  __syncthreads();
  double sv_sorted = 0.0;
  if (tid < n) sv_sorted = S.s[S.perm[tid] & 31];
  __syncthreads();
  if (tid < n) S.s[tid] = sv_sorted;
  for (int i = tid; i < 32 * 32; i += NTU_CTA) { S.V[i] = S.A[i]; }
  __syncthreads();
  for (int i = tid; i < 32 * 32; i += NTU_CTA) { S.A[i] = S.W[i]; }
  __syncthreads();
  if (phase) cta_svd_phase(S, m, n);
}

// Square n x n case with the phase convention.
__device__ inline void cta_svd_small(SvdSmem& S, int n) { cta_svd_cols(S, n, n, 1); }

// --------------------------------------- Hermitian tridiagonalisation
// A (n x n complex Hermitian, column-major, leading dim n, global memory) is
// reduced to a real symmetric tridiagonal T = Q^H A Q with
// Q = H_0 H_1 ... H_{n-2}.  Reflector j acts on rows j+1..n-1; its vector is
// v = [1; A[j+2:, j]] and its factor tau[j].  d[0..n) and e[0..n-1) receive T.
// p: scratch of n complex.  sred: >= 2*NTU_WARPS doubles.
__device__ inline void cta_hetrd(double2* __restrict__ A, int n, double* d, double* e,
                                 double2* tau, double2* p, double* sred) {
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
  for (int j = 0; j < n - 1; ++j) {
    const int m = n - j - 1;                 // length of the reflected part
    double2* col = A + (size_t)j * n + j + 1;   // A[j+1:, j]
    Reflector R = cta_reflector(col, m, sred);
    __syncthreads();
    for (int i = 1 + tid; i < m; i += NTU_CTA) col[i] = cmul(col[i], R.scale);
    if (tid == 0) {
      e[j] = R.beta; tau[j] = R.tau; d[j] = A[(size_t)j * n + j].x;
      col[0] = make_double2(1.0, 0.0);      // v[0] = 1 stored temporarily
    }
    __syncthreads();
    if (R.tau.x != 0.0 || R.tau.y != 0.0) {
      double2* A22 = A + (size_t)(j + 1) * n + j + 1;
      // p_i = tau * sum_k A22[i,k] v_k = tau * sum_k conj(A22[k,i]) v_k
      for (int i = wid; i < m; i += NTU_WARPS) {
        const double2* ci = A22 + (size_t)i * n;
        double2 acc = cz();
        for (int k = lid; k < m; k += 32) acc = cfmac(ci[k], col[k], acc);
        acc = warp_sum2(acc);
        if (lid == 0) p[i] = cmul(R.tau, acc);
      }
      __syncthreads();
      // w = p - (1/2) conj(tau) (v^H p) v
      double2 vp = cz();
      for (int i = tid; i < m; i += NTU_CTA) vp = cfmac(col[i], p[i], vp);
      vp = block_sum2(vp, sred);
      double2 f = cscale(cmul(cconj(R.tau), vp), 0.5);
      for (int i = tid; i < m; i += NTU_CTA) p[i] = cfms(f, col[i], p[i]);
      __syncthreads();
      // A22 -= v w^H + w v^H
      for (int idx = tid; idx < m * m; idx += NTU_CTA) {
        int k = idx % m, i = idx / m;          // row k, column i
        double2 a = A22[(size_t)i * n + k];
        double2 vk = col[k], wk = p[k], vi = col[i], wi = p[i];
        a = cfmsc(vk, wi, a);
        a = cfmsc(wk, vi, a);
        A22[(size_t)i * n + k] = a;
      }
      __syncthreads();
    }
  }
  if (tid == 0) d[n - 1] = A[(size_t)(n - 1) * n + n - 1].x;
  __syncthreads();
}

// b <- Q^H b (conj == true) or b <- Q b, with Q from cta_hetrd.
__device__ inline void cta_apply_q(const double2* __restrict__ A, int n, const double2* tau,
                                   double2* b, bool adjoint, double* sred) {
  const int tid = threadIdx.x;
  for (int jj = 0; jj < n - 1; ++jj) {
    int j = adjoint ? jj : (n - 2 - jj);
    double2 t = tau[j];
    if (t.x == 0.0 && t.y == 0.0) continue;
    const double2* v = A + (size_t)j * n + j + 1;   // v[0] = 1 implicitly
    int m = n - j - 1;
    double2* bb = b + j + 1;
    double2 s = cz();
    for (int i = tid; i < m; i += NTU_CTA) s = cfmac(i == 0 ? make_double2(1.0, 0.0) : v[i], bb[i], s);
    s = block_sum2(s, sred);
    double2 f = adjoint ? cmul(cconj(t), s) : cmul(t, s);
    for (int i = tid; i < m; i += NTU_CTA) bb[i] = cfms(f, i == 0 ? make_double2(1.0, 0.0) : v[i], bb[i]);
    __syncthreads();
  }
}

// ------------------------------------ implicit symmetric tridiagonal QR
// Eigenvalues of the real symmetric tridiagonal (d, e) (e[k] couples k and
// k+1) by implicit QR sweeps with the Wilkinson shift.  A sweep on the
// unreduced block [lo, hi] applies plane rotations G(k, k+1; c, s),
// k = lo..hi-1, so that T <- G^T T G; the eigenvectors are the columns of
// Z = G_1 G_2 ... G_m.

// Deflate negligible couplings and find the trailing unreduced block.
// Returns false when every eigenvalue has converged.
__device__ inline bool qr_next_block(double* d, double* e, int& lo, int& hi) {
  const double eps = 2.220446049250313e-16;
  while (hi > 0) {
    for (int k = 0; k < hi; ++k)
      if (fabs(e[k]) <= eps * (fabs(d[k]) + fabs(d[k + 1]))) e[k] = 0.0;
    if (e[hi - 1] == 0.0) { --hi; continue; }
    lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    return true;
  }
  return false;
}

// One bulge-chasing sweep on [lo, hi]; rotation t (acting on k = lo + t) is
// returned in cbuf[t], sbuf[t].
__device__ inline void qr_sweep(double* d, double* e, int lo, int hi, double* cbuf, double* sbuf) {
  double a = d[hi - 1], b = e[hi - 1], cc = d[hi];
  double dl = 0.5 * (a - cc);
  double den = dl + copysign(hypot(dl, b), dl);
  double mu = (den != 0.0) ? cc - b * b / den : cc - fabs(b);
  double x = d[lo] - mu, z = e[lo];
  for (int k = lo; k < hi; ++k) {
    double r = hypot(x, z);
    double c, s;
    if (r == 0.0) { c = 1.0; s = 0.0; }
    else { c = x / r; s = -z / r; }
    if (k > lo) e[k - 1] = r;
    double dk = d[k], dk1 = d[k + 1], ek = e[k];
    double cs = c * s;
    d[k] = c * c * dk - 2.0 * cs * ek + s * s * dk1;
    d[k + 1] = s * s * dk + 2.0 * cs * ek + c * c * dk1;
    e[k] = cs * (dk - dk1) + (c * c - s * s) * ek;
    if (k + 1 < hi) {
      double ek1 = e[k + 1];
      z = -s * ek1;
      e[k + 1] = c * ek1;
      x = e[k];
    }
    cbuf[k - lo] = c;
    sbuf[k - lo] = s;
  }
}

// Single-thread driver that appends every rotation to a log and applies
// Z^T to y on the fly.  Returns 0, or ST_NUMERIC on non-convergence or log
// overflow.
struct RotLog { double* c; double* s; int* k; int cap; int count; };

__device__ inline int tridiag_qr(double* d, double* e, int n, RotLog& log, double2* y) {
  log.count = 0;
  int lo = 0, hi = n - 1, iters = 0;
  while (qr_next_block(d, e, lo, hi)) {
    if (++iters > 40 * n) return ST_NUMERIC;
    int len = hi - lo;
    if (log.count + len > log.cap) return ST_NUMERIC;
    double* cb = log.c + log.count;
    double* sb = log.s + log.count;
    qr_sweep(d, e, lo, hi, cb, sb);
    for (int t = 0; t < len; ++t) {
      int k = lo + t;
      log.k[log.count + t] = k;
      if (y) {
        double c = cb[t], s = sb[t];
        double2 yk = y[k], yk1 = y[k + 1];
        y[k] = make_double2(c * yk.x - s * yk1.x, c * yk.y - s * yk1.y);
        y[k + 1] = make_double2(s * yk.x + c * yk1.x, s * yk.y + c * yk1.y);
      }
    }
    log.count += len;
  }
  return 0;
}

// CTA driver that accumulates Z explicitly (row-major n x n, global): thread
// 0 runs each sweep into the shared chain (2n doubles), then every thread
// applies the chain to its own rows of Z.  Returns 0 or ST_NUMERIC.
__device__ inline int cta_tridiag_qr_z(double* d, double* e, int n, double* Z, double* chain,
                                       int* shared_state) {
  const int tid = threadIdx.x;
  for (size_t idx = tid; idx < (size_t)n * n; idx += NTU_CTA)
    Z[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  int lo = 0, hi = n - 1, iters = 0;   // meaningful in thread 0 only
  __syncthreads();
  while (true) {
    if (tid == 0) {
      int st = 0, more = qr_next_block(d, e, lo, hi) ? 1 : 0;
      if (more && ++iters > 40 * n) { st = ST_NUMERIC; more = 0; }
      if (more) qr_sweep(d, e, lo, hi, chain, chain + n);
      shared_state[0] = more; shared_state[1] = lo; shared_state[2] = hi - lo;
      shared_state[3] = st;
    }
    __syncthreads();
    if (!shared_state[0]) break;
    const int l0 = shared_state[1], len = shared_state[2];
    for (int row = tid; row < n; row += NTU_CTA) {
      double* z = Z + (size_t)row * n;
      for (int t = 0; t < len; ++t) {
        int k = l0 + t;
        double c = chain[t], s = chain[n + t];
        double zk = z[k], zk1 = z[k + 1];
        z[k] = c * zk - s * zk1;
        z[k + 1] = s * zk + c * zk1;
      }
    }
    __syncthreads();
  }
  int st = shared_state[3];
  __syncthreads();
  return st;
}

// ------------------------------------------------------------ Cholesky
// In-place lower Cholesky factorisation of (A - shift * I) for a Hermitian A
// (column-major, leading dimension n, lower triangle referenced).  Returns 1
// if every pivot was positive and finite (the shifted matrix is numerically
// positive definite), 0 otherwise.  `flag`: one shared int.
__device__ inline int cta_cholesky(double2* __restrict__ A, int n, double shift, int* flag) {
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
  if (tid == 0) *flag = 1;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    double piv = A[(size_t)j * n + j].x - shift;
    if (!(piv > 0.0) || !isfinite(piv)) { if (tid == 0) *flag = 0; break; }
    double sp = sqrt(piv), rp = 1.0 / sp;
    double2* cj = A + (size_t)j * n;
    __syncthreads();
    if (tid == 0) cj[j] = make_double2(sp, 0.0);
    for (int i = j + 1 + tid; i < n; i += NTU_CTA) cj[i] = cscale(cj[i], rp);
    __syncthreads();
    for (int k = j + 1 + wid; k < n; k += NTU_WARPS) {
      const double2 lk = cj[k];
      double2* ck = A + (size_t)k * n;
      for (int i = k + lid; i < n; i += 32) ck[i] = cfmsc(cj[i], lk, ck[i]);
    }
    __syncthreads();
  }
  __syncthreads();
  int ok = *flag;
  __syncthreads();
  return ok;
}

// cta_cholesky in double-FP32 arithmetic (A column-major as FP32 pairs,
// (re_hi, im_hi, re_lo, im_lo), lower triangle, no shift): the same
// right-looking steps, with each pivot's square root and reciprocal taken
// in FP64 from its exact double value.  Returns 1 if every pivot was positive
// and finite.  Used as the positive-definiteness certificate where the
// metric itself carries FP32 rounding.  col: n float4 of shared memory (the
// current column, staged for the trailing update).
__device__ inline int cta_cholesky_df(float4* __restrict__ A, int n, int* flag,
                                      float4* __restrict__ col) {
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
  if (tid == 0) *flag = 1;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const float4 dj = A[(size_t)j * n + j];
    const double piv = (double)dj.x + (double)dj.z;
    if (!(piv > 0.0) || !isfinite(piv)) { if (tid == 0) *flag = 0; break; }
    const double sp = sqrt(piv), rp = 1.0 / sp;
    const float rh = (float)rp, rl = (float)(rp - (double)rh);
    const float4 rdf = make_float4(rh, 0.f, rl, 0.f);
    float4* cj = A + (size_t)j * n;
    __syncthreads();
    if (tid == 0) {
      const float sh = (float)sp;
      cj[j] = make_float4(sh, 0.f, (float)(sp - (double)sh), 0.f);
    }
    // the scaled column j, also staged in shared memory for the update
    for (int i = j + 1 + tid; i < n; i += NTU_CTA) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      df_cmac<false>(acc, cj[i], rdf);
      cj[i] = acc;
      col[i] = acc;
    }
    __syncthreads();
    // trailing update, a warp per column k, four independent rows per lane
    // and iteration (one load-modify-store at a time left this latency-bound)
    for (int k = j + 1 + wid; k < n; k += NTU_WARPS) {
      const float4 lk = col[k];
      float4* ck = A + (size_t)k * n;
      for (int i0 = k + lid; i0 < n; i0 += 128) {
        float4 acc[4], ci[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          if (i < n) { acc[u] = ck[i]; ci[u] = col[i]; }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          if (i < n) {
            df_cmac<true>(acc[u], lk, make_float4(-ci[u].x, -ci[u].y, -ci[u].z, -ci[u].w));   // -= c_i conj(l_k)
            ck[i] = acc[u];
          }
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  int ok = *flag;
  __syncthreads();
  return ok;
}

// Solve (L L^H) x = b in place with the factor from cta_cholesky, by one
// warp (no CTA barriers): lane l owns the entries i = l (mod 32) of b, which
// lives in shared memory.  Must be called by all 32 lanes of one warp.
__device__ inline void warp_cholesky_solve(const double2* __restrict__ L, int n, double2* b) {
  const int lid = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {           // L y = b
    if ((j & 31) == lid) b[j] = cscale(b[j], 1.0 / L[(size_t)j * n + j].x);
    __syncwarp();
    const double2 yj = b[j];
    const double2* cj = L + (size_t)j * n;
    for (int i = j + 1 + ((lid - j - 1) & 31); i < n; i += 32) b[i] = cfms(cj[i], yj, b[i]);
    __syncwarp();
  }
  for (int j = n - 1; j >= 0; --j) {      // L^H x = y
    if ((j & 31) == lid) b[j] = cscale(b[j], 1.0 / L[(size_t)j * n + j].x);
    __syncwarp();
    const double2 xj = b[j];
    for (int i = lid; i < j; i += 32) b[i] = cfmsc(xj, L[(size_t)i * n + j], b[i]);
    __syncwarp();
  }
}

// Solve (L L^H) x = b in place with the factor from cta_cholesky.
__device__ inline void cta_cholesky_solve(const double2* __restrict__ L, int n, double2* b) {
  const int tid = threadIdx.x;
  for (int j = 0; j < n; ++j) {           // L y = b
    __syncthreads();
    double2 yj = cscale(b[j], 1.0 / L[(size_t)j * n + j].x);
    __syncthreads();
    if (tid == 0) b[j] = yj;
    const double2* cj = L + (size_t)j * n;
    for (int i = j + 1 + tid; i < n; i += NTU_CTA) b[i] = csub(b[i], cmul(cj[i], yj));
  }
  for (int j = n - 1; j >= 0; --j) {      // L^H x = y
    __syncthreads();
    double2 xj = cscale(b[j], 1.0 / L[(size_t)j * n + j].x);
    __syncthreads();
    if (tid == 0) b[j] = xj;
    for (int i = tid; i < j; i += NTU_CTA) b[i] = csub(b[i], cmul(cconj(L[(size_t)i * n + j]), xj));
  }
  __syncthreads();
}

// u <- Z u (rotations replayed in reverse), single thread.
__device__ inline void rotlog_apply_z(const RotLog& log, double2* u) {
  for (int t = log.count - 1; t >= 0; --t) {
    int k = log.k[t];
    double c = log.c[t], s = log.s[t];
    double2 a = u[k], b = u[k + 1];
    u[k] = make_double2(c * a.x + s * b.x, c * a.y + s * b.y);
    u[k + 1] = make_double2(-s * a.x + c * b.x, -s * a.y + c * b.y);
  }
}

}  // namespace ntu
