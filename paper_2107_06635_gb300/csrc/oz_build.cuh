// Tensor-core build of the ALS reduced metric (Fig. 5(b)) with exact
// integer slicing, for K = D r = 16 or 32 on the mixed contexts.
//
// Per half sweep the reduced metric is g_A = (1 x F)^H g (1 x F) with F the
// fixed K x D factor (M_B on the A step, M_A on the B step).  Its first and
// larger stage, T_f = g[:, f-block] F for every column block f of g, is a
// product of an n_g x K matrix with a K x D one per block: here it runs on
// the tensor cores without losing precision beyond ~2^-48, so the result
// matches the double-FP32 lane arithmetic of the other path.
//
// Slicing (an error-free splitting in the manner of Ozaki, Ogita, Oishi and
// Rump's exact matrix products): each row segment of g (16 complex entries
// of one row in one column block) is scaled by a power of two 2^-e so that
// its entries lie in (-1, 1), and written as six BF16 slices of integer
// digits, x = sum_i d_i 2^-8(i+1) + O(2^-49) with |d_i| <= 255 (exact in
// BF16's 8-bit significand).  F's columns are sliced the same way with their
// own exponents.  A product of two slices over the K = 32 real terms of a
// complex dot product is an integer below 2^21, and the at most six slice
// pairs (i, j) of one level l = i + j sum to less than 2^24, so each level's
// FP32 tensor-core accumulator is exact.  Levels 0..5 are kept (the dropped
// ones are below 2^-48 of the row maximum); they are combined in double-FP32
// and scaled back, which is where the only rounding happens.
//
// The complex product is one real GEMM: A rows are [Re g (16) | Im g (16)],
// B rows (output columns) are [Re F | -Im F] for Re T and [Im F | Re F] for
// Im T.  One M = 128 row tile of A (8 row blocks f1 of g) times all of B's
// slices needs 6 MMAs (A slice i against B slices 0..5-i, N = (6-i) 16,
// accumulated into TMEM columns 16 i ..: column block l holds level l), two
// K = 16 steps each.  The A slices come by TMA (128-byte swizzle, two slices
// per 128-byte row, double-buffered), B is written into shared memory by the
// CTA once per half sweep.  The epilogue (warps 0-3, one TMEM lane per
// thread) combines the six levels of each output into double-FP32 and
// stages the tile of T in shared memory; the second stage, the D x D blocks
// F^H T, stays on the FP32 lanes in double-FP32 (als_reduced_df's second
// loop).  Only blocks f1 >= f are built (g_A is Hermitian), so of the 32
// row tiles of a half sweep 24 are computed.
#pragma once
#include <cuda_bf16.h>

#include "ntu_dev.cuh"
#include "tc_sm103.cuh"

namespace ntu {

constexpr int OZ_SLICES = 6;
constexpr int OZ_LEVEL_COLS = 16;           // accumulator columns per level (2 D <= 16)
constexpr int OZ_TMEM_COLS = 128;           // 6 levels x 16 columns, rounded up
constexpr int OZ_BOX_BYTES = 128 * 128;     // 128 rows x 64 BF16
constexpr int OZ_B_ROWS = OZ_SLICES * OZ_LEVEL_COLS;   // 96
constexpr long long OZ_WAIT = 1ll << 26;
constexpr int OZ_POLLS = 1 << 16;           // polls of up to 20 us each: about a second

// Geometry of the build for K = 16 or 32 (n_g = K^2 rows of g, 128-row
// tiles): a 128-byte box row holds spb = 32 / K slices of a row segment
// (2 K reals each), so a tile takes boxes = 6 / spb boxes and each slice
// K / 8 MMA K-steps; a tile covers bpt = 128 / K row blocks f1, a column
// block f has T = n_g / 128 tiles, of which those holding a block f1 >= f
// are built (ntiles per half sweep).
struct OzGeo {
  int K, ng, spb, boxes, ksteps, bpt, T, ntiles;
  long long rows_side;       // box rows of one ALS step's slices
};
__host__ __device__ inline OzGeo oz_geo(int K) {
  OzGeo g;
  g.K = K; g.ng = K * K; g.spb = 32 / K; g.boxes = OZ_SLICES / g.spb; g.ksteps = K / 8;
  g.bpt = 128 / K; g.T = g.ng / 128;
  g.ntiles = 0;
  for (int f = 0; f < K; ++f) g.ntiles += g.T - f / g.bpt;
  g.rows_side = (long long)K * g.T * g.boxes * 128;
  return g;
}
__host__ __device__ inline bool oz_supported(int K) { return K == 16 || K == 32; }

// Rows of the slice array of one item: [side][f][t][box][128 rows], each row
// 64 BF16 = spb slices x [Re (K) | Im (K)].
__device__ __forceinline__ long long oz_row(const OzGeo& G, int side, int f, int t, int box) {
  return (long long)side * G.rows_side + ((long long)(f * G.T + t) * G.boxes + box) * 128;
}

// Tile tau of a half sweep -> column block f and row tile t (f major, t
// from the first tile holding a block f1 >= f): the bpt columns blocks f of
// group b = f / bpt each have T - b tiles.
__device__ __forceinline__ void oz_tile_ft(const OzGeo& G, int tau, int& f, int& t) {
  int b = 0, cum = 0;
  while (b < G.T - 1 && tau >= cum + G.bpt * (G.T - b)) { cum += G.bpt * (G.T - b); ++b; }
  const int w = G.T - b, rem = tau - cum;
  f = b * G.bpt + rem / w;
  t = b + rem % w;
}

__device__ __forceinline__ void oz_fence_proxy_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void oz_fence_proxy_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Fixed-point digits from FP64 bit patterns, with integer operations only
// (FP64 arithmetic, and 64-bit integer <-> float conversions, issue at a
// small fraction of the FP32 rate on this GPU).
//
// oz_bexp(v): an exponent e with |v| < 2^e (from v's exponent field; 0
// for zero and subnormal values, which are below every scale used here).
__device__ __forceinline__ int oz_bexp(double v) {
  const int ef = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
  return ef == 0 ? -100000 : ef - 1022;
}

// X = v 2^(48 - e) rounded to an integer (|X| < 2^48 when |v| < 2^e):
// v = m 2^(ef - 1075) with the 53-bit significand m, so X = m shifted by
// ef - 1027 - e (rounded half away from zero on a right shift).
__device__ __forceinline__ long long oz_fixed(double v, int e) {
  const long long b = __double_as_longlong(v);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0) return 0;
  const long long m = (b & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;
  const int sh = ef - 1027 - e;
  long long x;
  if (sh >= 0) x = m << sh;
  else if (sh > -54) x = (m + (1ll << (-sh - 1))) >> (-sh);
  else x = 0;
  return b < 0 ? -x : x;
}

// BF16 bit pattern of digit i (0 = most significant) of X: the signed
// integer sign(X) * byte (5 - i) of |X|, |d| <= 255, which BF16 holds
// exactly (8-bit significand); built from the bits directly.
__device__ __forceinline__ uint32_t oz_digit_bits(long long X, int i) {
  const unsigned long long mg = (unsigned long long)(X < 0 ? -X : X);
  const uint32_t d = (uint32_t)((mg >> (40 - 8 * i)) & 255u);
  if (d == 0) return 0u;
  const int p = 31 - __clz((int)d);                     // leading one, 0..7
  const uint32_t bits = ((uint32_t)(127 + p) << 7) | ((d << (7 - p)) & 0x7fu);
  return X < 0 ? (bits | 0x8000u) : bits;
}

// Slices of g for both ALS steps of every item (one launch over the batch,
// before the ALS kernel): gsl rows as oz_row, gexp[item][side][f][R] the
// segment exponents (relative to the unscaled g).  Side 1 reads g with kA
// and kB swapped in rows and columns (the B step's view).  Thread task:
// one 8-value group (real or imaginary part of 8 consecutive entries) of
// one row segment; the K / 4 groups of a segment are adjacent lanes, which
// agree on the exponent by shuffles.  Each task writes its 16-byte chunk of
// all six slices.  KK = K = D r (16 or 32).
template <int KK>
__global__ void __launch_bounds__(NTU_CTA) k_oz_slice(int n, const double2* __restrict__ g,
                                                      __nv_bfloat16* __restrict__ gsl,
                                                      short* __restrict__ gexp) {
  constexpr int K = KK;
  const OzGeo G = oz_geo(K);
  const int ng = G.ng, gps = K / 4;                    // groups per segment: 4 or 8
  const long long tasks = (long long)n * 2 * K * ng * gps;
  for (long long task = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       task - threadIdx.x < tasks; task += (long long)gridDim.x * blockDim.x) {
    const bool live = task < tasks;
    const long long tk = live ? task : 0;
    const int grp = (int)(tk % gps);
    const long long seg = tk / gps;
    const long long item = seg / (2LL * K * ng);
    const int side = (int)((seg / ((long long)K * ng)) % 2), f = (int)((seg / ng) % K),
              R = (int)(seg % ng);
    const double2* gi = g + item * (long long)ng * ng;
    const double2* rowp = side == 0 ? gi + (size_t)R * ng + f * K
                                    : gi + (size_t)((R % K) * K + R / K) * ng + f;
    const int cs = side == 0 ? 1 : K;
    const int part = grp / (K / 8), c0 = (grp % (K / 8)) * 8;
    double x[8];
    int e = -100000;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double2 v = rowp[(c0 + k) * cs];
      x[k] = part ? v.y : v.x;
    }
    // the segment exponent covers all 2 K reals: the other groups' maxima
    // come from the partner lanes
#pragma unroll
    for (int k = 0; k < 8; ++k) e = max(e, oz_bexp(x[k]));
    for (int o = 1; o < gps; o <<= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (e < -1000) e = 0;                                // an all-zero segment
    if (!live) continue;
    if (grp == 0) gexp[(item * 2 + side) * (long long)K * ng + f * ng + R] = (short)e;
    long long X[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) X[k] = oz_fixed(x[k], e);
    const int t = R >> 7, r = R & 127;
    __nv_bfloat16* base = gsl + item * 2 * G.rows_side * 64;
#pragma unroll
    for (int i = 0; i < OZ_SLICES; ++i) {
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 8; k += 2)
        w[k >> 1] = oz_digit_bits(X[k], i) | (oz_digit_bits(X[k + 1], i) << 16);
      const long long row = oz_row(G, side, f, t, i / G.spb) + r;
      *reinterpret_cast<uint4*>(base + row * 64 + (i % G.spb) * 2 * K + grp * 8) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Shared-memory pieces of the build, carved from the ALS CTA's SVD work
// arrays (free during a build) from the first 1024-byte boundary on: two A
// box buffers, the B operand and F in double-FP32, 48 KB at K = 32 (the
// arrays are followed by 1 KB of slack for the alignment).  The column
// exponents, the failure flag and the
// mbarriers take the CTA's reduction scratch (unused during a build); the
// barriers are initialised afresh for every build (all their phases
// complete within it), so the permanent shared state does not grow.
struct OzSmem {
  unsigned char* abuf;     // 2 x OZ_BOX_BYTES
  unsigned char* bop;      // OZ_B_ROWS x 128 bytes
  float4* fdf;             // K x D
  int* eq;                 // D column exponents
  int* dead;               // a tensor-core wait ran out
  uint64_t* bar;           // A box full [2], A box free [2], accumulator ready, done
};

__device__ __forceinline__ OzSmem oz_smem(void* region, double* scratch) {
  OzSmem s;
  unsigned char* p = (unsigned char*)(((uintptr_t)region + 1023) & ~(uintptr_t)1023);
  s.abuf = p;
  s.bop = p + 2 * OZ_BOX_BYTES;
  s.fdf = reinterpret_cast<float4*>(s.bop + OZ_B_ROWS * 128);
  s.eq = reinterpret_cast<int*>(scratch);
  s.dead = s.eq + 8;
  s.bar = reinterpret_cast<uint64_t*>(scratch + 5);
  return s;
}

// Bytes of the build's shared pieces in the SVD arrays at the largest K.
constexpr size_t OZ_SMEM_BYTES = 2 * OZ_BOX_BYTES + OZ_B_ROWS * 128 + 32 * 8 * sizeof(float4);

// B operand of one half sweep from F (K x D, FP64 complex): row
// l * 16 + 2 q + part holds slice l of output column (q, part) over the 2 K
// real K positions, written with the 128-byte swizzle the MMA descriptor
// expects (16-byte chunk c of row n at chunk c ^ (n & 7)).  Also F in
// double-FP32 for the second stage.
static __device__ void oz_fill_b(const OzSmem& s, const double2* F, int K, int D) {
  const int tid = threadIdx.x, cpr = K / 4;            // used chunks per row
  for (int i = tid; i < K * D; i += NTU_CTA) s.fdf[i] = df_split(F[i]);
  if (tid < D) {
    int e = -100000;
    for (int c = 0; c < K; ++c) e = max(e, max(oz_bexp(F[c * D + tid].x), oz_bexp(F[c * D + tid].y)));
    s.eq[tid] = e < -1000 ? 0 : e;
  }
  __syncthreads();
  for (int it = tid; it < OZ_B_ROWS * cpr; it += NTU_CTA) {
    const int n = it / cpr, ch = it % cpr;
    const int lvl = n >> 4, m = n & 15, q = m >> 1, part = m & 1;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (q < D) {
      const int e = s.eq[q];
      // K position kpos = ch * 8 + k: first half c = kpos (Re F or Im F),
      // second half c = kpos - K (-Im F or Re F)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int kpos = ch * 8 + k, c = kpos < K ? kpos : kpos - K;
        const double2 fv = F[c * D + q];
        long long X;
        if (kpos < K) X = oz_fixed(part ? fv.y : fv.x, e);
        else X = part ? oz_fixed(fv.x, e) : -oz_fixed(fv.y, e);
        w[k >> 1] |= oz_digit_bits(X, lvl) << (16 * (k & 1));
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(s.bop + n * 128 + ((ch ^ (n & 7)) << 4));
    *dst = make_uint4(w[0], w[1], w[2], w[3]);
  }
  oz_fence_proxy_smem();
  __syncthreads();
}

}  // namespace ntu
