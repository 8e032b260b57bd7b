// Fused t1 -> t2 of the half environment (Fig. 4(c,d)) on tcgen05 for the
// NTU_MIXED_BF16X3 precision.
//
// For one item and one bond-index pair (k, k') the double isometry block
//   T1[(u,n),(u',n')] = sum_{p,e'} Y[p,e',u,n,k] conj(Q[p,e',u',n',k'])
// and the top-edge contraction
//   T2[(ht,ht'),(n,n')] = sum_{u,u'} E_top[ht,u,ht',u'] T1[(u,n),(u',n')]
// are two chained GEMMs.  The first runs on the tensor cores into TMEM, its
// result is split into BF16 hi/lo and written by the epilogue warps straight
// into shared memory as the (128-byte swizzled, K-major) B operand of the
// second, so T1 never leaves the SM; only T2 goes to HBM, as the split B
// operand of h (rows (k,k',ht,ht'), complex columns (n',n) with the real
// parts of a row's columns first and the imaginary parts krpE/2 later).
//
// Complex products are real GEMMs as in k_tc.cu: A doubled (Re / Im rows 64
// apart in a 128-row tile), three split products hi*hi + hi*lo + lo*hi
// accumulated in FP32.  GEMM1 (A = Y, B = conj(Q), from TMA) keeps (re, im)
// interleaved along K; GEMM2 has K planar (all Re factors, then all Im) and
// takes its A operand, E_top, from tensor memory, where epilogue 2 copies it
// from global memory once per item (one 128-byte row segment per thread and
// K chunk).
//
// One persistent CTA per SM takes a contiguous range of (item, k, k') units.
// Warp 0 issues TMA (the Y block once per k, the conj(Q) block per unit,
// double-buffered), warp 1 issues the MMAs (GEMM1 of unit i, then GEMM2 of
// unit i-1), warps 2-9 turn accumulator 1 into the B operand of GEMM2 (two
// buffers), warps 10-17 turn accumulator 2 into output rows in a swizzled
// shared staging block that one thread stores with TMA.
//
// At D = 8 the units (k, k') and (k, k'+1) form a pair: epilogue 1 writes
// both into one 128-row operand buffer (two such buffers) and GEMM2 of the
// pair is one N = 128 product.  This halves GEMM2's MMA instructions, whose
// issue (about 77 cycles each, whatever N), not the tensor pipe, sets the
// kernel's pace.
//
// Both epilogues write 16-byte chunks: the planar K of GEMM2 puts the eight
// u' values of one (u, n') next to each other, and the planar T2 the
// sixteen columns a thread holds.  Every wait is bounded; every role leaves
// its loop on a timeout and the epilogue groups leave together.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ntu_dev.cuh"
#include "ntu_impl.h"
#include "tc_sm103.cuh"

namespace ntu {

namespace {
constexpr int EPI = 256;                       // threads of each epilogue group
constexpr int T12_THREADS = 64 + 2 * EPI;
constexpr long long T12_WAIT = 1ll << 28;
constexpr int T12_SLEEP_POLLS = 1 << 17;       // x <= 20 us: about 2.6 s
constexpr int A_TILE = 128 * 128;            // 128 rows x 64 BF16
constexpr int B_TILE = 64 * 128;             // 64 rows x 64 BF16
constexpr int OFF_A1 = 0;                     // 2 A tiles: Y hi, lo
constexpr int OFF_B1 = OFF_A1 + 2 * A_TILE;   // 2 buffers x 2 B tiles: conj(Q) hi, lo
// GEMM2 B operand, T1 hi0, hi1, lo0, lo1: 2 buffers of 4 64-row tiles, or
// of 4 128-row tiles for unit pairs
constexpr int OFF_B2 = OFF_B1 + 4 * B_TILE;
constexpr int B2_BYTES = 16 * B_TILE;
constexpr int STG_BOX = 64 * 128;             // one output box: 64 rows x 64 BF16
constexpr int OFF_STG = OFF_B2 + B2_BYTES;    // output staging: up to 4 boxes (hi Re/Im, lo Re/Im)
constexpr int OFF_BAR = OFF_STG + 4 * STG_BOX;
// TMEM columns: accumulator 1 (two buffers of 64) 0-127, accumulator 2
// (two buffers of 64, or of 128 for unit pairs) from 128, E_top as the A
// operand of GEMM2: hi halves from 384, lo halves from 448
constexpr uint32_t TM_COLS = 512, TM_A2H = 384, TM_A2L = 448;
constexpr size_t T12_SMEM = (size_t)OFF_BAR + 512 + 1024;
static_assert(T12_SMEM <= 227 * 1024, "shared memory budget");

// Byte offset of BF16 element w (0..63) of row r in a K-major tile with
// 128-byte rows written with the 128-byte swizzle (what TMA writes and the
// MMA descriptor of tc::sdesc_k128 expects): the 16-byte chunk index is
// XORed with the row index modulo 8.
__device__ __forceinline__ uint32_t swz(int r, int w) {
  return (uint32_t)(r * 128 + ((((w >> 3) ^ (r & 7))) << 4) + ((w & 7) << 1));
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
}  // namespace

struct T12Args {
  int D, K;
  int nchunk;           // 64-wide K chunks of GEMM2 (krpE / 64)
  int krpY, krpE;
  int k1;               // 16-wide K steps of GEMM1 that hold data: ceil(2 d_p D / 16)
  long long units;      // items * K * K
  const __nv_bfloat16* E;   // E_top split: per item rows of 2 krpE (hi, then lo)
  long long e_item;         // elements per item of E
  int* err;
};

// DT = 8: bond dimension fixed at compile time (every index of the epilogues
// folds into constants); DT = 0: any D <= 8 at run time.
template <int DT>
__global__ void __launch_bounds__(T12_THREADS, 1) k_t12(const __grid_constant__ CUtensorMap mA1,
                                                      const __grid_constant__ CUtensorMap mB1,
                                                      const __grid_constant__ CUtensorMap mT2,
                                                      T12Args a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = (uint64_t*)(sm + OFF_BAR);
  uint64_t *a1_full = bar + 2, *a1_empty = bar + 3;
  uint64_t *q_full = bar + 4, *q_empty = bar + 6;             // [2]
  uint64_t *c1_full = bar + 8, *c1_empty = bar + 10;          // accumulator 1 [2]
  uint64_t *b2_full = bar + 12, *b2_empty = bar + 14;         // GEMM2 B operand [2]
  uint64_t *c2_full = bar + 16, *c2_empty = bar + 18;         // accumulator 2 [2]
  uint64_t* done = bar + 20;
  uint32_t* tmem_slot = (uint32_t*)(bar + 21);
  uint64_t* a2t_full = bar + 22;                               // E_top copied into TMEM
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = DT ? DT : a.D, K = a.K, D2 = D * D, KK = K * K;
  // D = 8: units (k, k') and (k, k'+1) are paired (K = 8 r is even): GEMM2
  // of a pair is one N = 128 product, from one 128-row operand buffer
  constexpr bool PAIR = DT == 8;
  // contiguous range of units for this CTA (whole pairs when paired)
  const long long ug = PAIR ? a.units / 2 : a.units;
  const long long u0 = (PAIR ? 2 : 1) * (ug * blockIdx.x / gridDim.x);
  const long long u1 = (PAIR ? 2 : 1) * (ug * (blockIdx.x + 1) / gridDim.x);
  // padding of the generated operand and of the output staging must read
  // as zero: clear both once (generic stores, then a proxy fence)
  for (int i = tid; i < (B2_BYTES + 4 * STG_BOX) / 16; i += T12_THREADS)
    reinterpret_cast<uint4*>(sm + OFF_B2)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async();
  if (tid == 0) {
    tc::mbar_init(a1_full, 1); tc::mbar_init(a1_empty, 1);
    tc::mbar_init(a2t_full, EPI / 32);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&q_full[b], 1); tc::mbar_init(&q_empty[b], 1);
      tc::mbar_init(&c1_full[b], 1); tc::mbar_init(&c1_empty[b], EPI / 32);
      tc::mbar_init(&b2_full[b], 1); tc::mbar_init(&b2_empty[b], 1);
      tc::mbar_init(&c2_full[b], 1); tc::mbar_init(&c2_empty[b], EPI / 32);
    }
    tc::mbar_init(done, 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, TM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: per unit the Y block if (item, k) changed, then the
      // conj(Q) block
      int a1z = -1, a1k = -1;
      long long a1n = 0, qn = 0, i = 0;
      // unit u = (z, k, kp): kept incrementally (no 64-bit division per unit)
      int z = (int)(u0 / KK), k = (int)(u0 % KK) / K, kp = (int)(u0 % KK) % K;
      for (long long u = u0; u < u1; ++u, ++i, kp = kp + 1 < K ? kp + 1 : 0,
                     k = kp ? k : (k + 1 < K ? k + 1 : 0), z = (kp || k) ? z : z + 1) {
        if (z != a1z || k != a1k) {
          if (a1n > 0 && !tc::mbar_wait(a1_empty, (uint32_t)((a1n - 1) & 1), T12_WAIT)) {
            raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
            break;
          }
          tc::mbar_expect_tx(a1_full, 2 * A_TILE);
          tc::tma_load_3d(sm + OFF_A1, &mA1, a1_full, 0, k * 128, z);
          tc::tma_load_3d(sm + OFF_A1 + A_TILE, &mA1, a1_full, a.krpY, k * 128, z);
          ++a1n; a1z = z; a1k = k;
        }
        const int qb = (int)(i & 1);
        const long long qu = i >> 1;
        if (qu > 0 && !tc::mbar_wait(&q_empty[qb], (uint32_t)((qu - 1) & 1), T12_WAIT)) {
          raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
          break;
        }
        unsigned char* qd = sm + OFF_B1 + qb * 2 * B_TILE;
        tc::mbar_expect_tx(&q_full[qb], 2 * B_TILE);
        tc::tma_load_3d(qd, &mB1, &q_full[qb], 0, kp * 64, z);
        tc::tma_load_3d(qd + B_TILE, &mB1, &q_full[qb], a.krpY, kp * 64, z);
        ++qn;
      }
      // no TMA copy may still be landing in shared memory when the CTA exits
      bool dr = true;
      if (a1n > 0) dr &= tc::mbar_wait(a1_full, (uint32_t)((a1n - 1) & 1), T12_WAIT);
      for (long long q = qn - 2 < 0 ? 0 : qn - 2; q < qn; ++q)
        dr &= tc::mbar_wait(&q_full[q & 1], (uint32_t)((q >> 1) & 1), T12_WAIT);
      if (!dr) raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: GEMM1 of unit i, then GEMM2 of unit i - 1
      const uint32_t id = tc::idesc_bf16_f32(128, 64);
      int a1z = -1, a1k = -1, a2z = -1;
      long long a1n = 0, a2n = 0, i = 0;
      bool ok = true;
      // unit u = (z, k, kp) kept incrementally; zp is the item of unit u - 1
      int z = (int)(u0 / KK), k = (int)(u0 % KK) / K, kp = (int)(u0 % KK) % K, zp = -1;
      for (long long u = u0; u <= u1 && ok; ++u, ++i) {
        if (u < u1) {
          if (z != a1z || k != a1k) {
            if (!tc::mbar_wait(a1_full, (uint32_t)(a1n & 1), T12_WAIT)) { ok = false; break; }
            ++a1n; a1z = z; a1k = k;
          }
          const int b = (int)(i & 1);
          const long long ub = i >> 1;
          if (ub > 0 && !tc::mbar_wait(&c1_empty[b], (uint32_t)((ub - 1) & 1), T12_WAIT)) { ok = false; break; }
          if (!tc::mbar_wait(&q_full[b], (uint32_t)(ub & 1), T12_WAIT)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t acc = tmem + (uint32_t)(b * 64);
          const uint64_t ah = tc::sdesc_k128(tc::smem_u32(sm + OFF_A1));
          const uint64_t al = tc::sdesc_k128(tc::smem_u32(sm + OFF_A1 + A_TILE));
          const uint64_t bh = tc::sdesc_k128(tc::smem_u32(sm + OFF_B1 + b * 2 * B_TILE));
          const uint64_t bl = tc::sdesc_k128(tc::smem_u32(sm + OFF_B1 + b * 2 * B_TILE + B_TILE));
          for (int kk4 = 0; kk4 < a.k1; ++kk4) {     // K beyond 2 d_p D is zero padding
            tc::mma_bf16(acc, ah + 2 * kk4, bh + 2 * kk4, id, kk4 != 0);
            tc::mma_bf16(acc, ah + 2 * kk4, bl + 2 * kk4, id, 1);
            tc::mma_bf16(acc, al + 2 * kk4, bh + 2 * kk4, id, 1);
          }
          tc::mma_commit(&q_empty[b]);
          tc::mma_commit(&c1_full[b]);
          // the Y block is released after the last unit that reads it (the
          // next unit starts a new k, or there is none)
          if (u + 1 >= u1 || kp == K - 1) tc::mma_commit(a1_empty);
        }
        if (u > u0 && (!PAIR || (i & 1) == 0)) {
          // GEMM2 of unit j = u - 1, or of pair j = i / 2 - 1 (units u - 2,
          // u - 1) into 128 accumulator columns; operand buffer j % 2
          const long long j = PAIR ? (i >> 1) - 1 : i - 1;
          const int zj = zp;
          const int b = (int)(j & 1);
          const long long ub = j >> 1;
          if (zj != a2z) {                      // E_top of the item is in TMEM
            if (!tc::mbar_wait(a2t_full, (uint32_t)(a2n & 1), T12_WAIT)) { ok = false; break; }
            ++a2n; a2z = zj;
          }
          if (!tc::mbar_wait(&b2_full[b], (uint32_t)(ub & 1), T12_WAIT)) { ok = false; break; }
          if (ub > 0 && !tc::mbar_wait(&c2_empty[b], (uint32_t)((ub - 1) & 1), T12_WAIT)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t acc = tmem + 128u + (uint32_t)(b * (PAIR ? 128 : 64));
          const uint32_t id2 = PAIR ? tc::idesc_bf16_f32(128, 128) : id;
          const int tstride = PAIR ? 2 * B_TILE : B_TILE;
          unsigned char* B2 = sm + OFF_B2 + b * (PAIR ? 8 : 4) * B_TILE;
          for (int c = 0; c < a.nchunk; ++c) {
            const uint32_t ah = tmem + TM_A2H + (uint32_t)(c * 32);
            const uint32_t al = tmem + TM_A2L + (uint32_t)(c * 32);
            const uint64_t bh = tc::sdesc_k128(tc::smem_u32(B2 + c * tstride));
            const uint64_t bl = tc::sdesc_k128(tc::smem_u32(B2 + (2 + c) * tstride));
#pragma unroll
            for (int kk4 = 0; kk4 < 4; ++kk4) {
              tc::mma_bf16_ts(acc, ah + 8 * kk4, bh + 2 * kk4, id2, (c | kk4) != 0);
              tc::mma_bf16_ts(acc, ah + 8 * kk4, bl + 2 * kk4, id2, 1);
              tc::mma_bf16_ts(acc, al + 8 * kk4, bh + 2 * kk4, id2, 1);
            }
          }
          tc::mma_commit(&b2_empty[b]);
          tc::mma_commit(&c2_full[b]);
        }
        zp = z;
        if (++kp == K) {
          kp = 0;
          if (++k == K) { k = 0; ++z; }
        }
      }
      if (!ok) raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
      // every MMA issued has retired before TMEM is released
      tc::mma_commit(done);
      if (!tc::mbar_wait(done, 0, T12_WAIT)) raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
    }
    __syncwarp();
  } else if (warp < 2 + EPI / 32) {
    // ---- epilogue 1: accumulator 1 (rows (u,n) Re / Im, columns
    // (n',u')) -> split B operand of GEMM2 in shared memory: row n' * D + n,
    // K planar, Re of (u,u') at u * D + u' and Im krpE/2 later.  With D = 8
    // a thread's eight values of one n' (u' = 0..7) are one 16-byte chunk of
    // hi and one of lo; the chunk of row n'*8 + n that holds (u, .) is the
    // 128-byte-swizzle slot u ^ n, so the 32 lanes of a warp (4 u x 8 n)
    // cover all eight slots four times: conflict-free quarter-warp phases.
    // warp w reads TMEM lanes 32 (w % 4) .. +31, columns slice * 32 .. +31
    const int et = tid - 64, quarter = warp & 3, row = quarter * 32 + lane;
    const int cs = ((warp - 2) >> 2) * 32;
    const int r = row & 63, im = row >> 6;
    const bool rv = r < D2;
    const int uu = rv ? r / D : 0, nn = rv ? r % D : 0;
    const int half = a.krpE / 2;
    long long i = 0;
    for (long long u = u0; u < u1; ++u, ++i) {
      const int b = (int)(i & 1);
      const long long ub = i >> 1;
      // one thread waits (suspended in hardware), the group meets at a
      // named barrier that also carries the outcome
      bool got = true;
      // operand buffer: slot s (the unit, or its pair) goes to buffer s % 2,
      // free once GEMM2 of slot s - 2 has completed
      const long long sl = PAIR ? i >> 1 : i;
      const int sb = (int)(sl & 1);
      const long long sub = sl >> 1;
      const bool first = !PAIR || b == 0, last = !PAIR || b == 1;
      if (et == 0) {
        got = tc::mbar_wait_sleep(&c1_full[b], (uint32_t)(ub & 1), T12_SLEEP_POLLS);
        if (got && first && sub > 0)
          got = tc::mbar_wait_sleep(&b2_empty[sb], (uint32_t)((sub - 1) & 1), T12_SLEEP_POLLS);
      }
      if (!tc::bar_and(1, EPI, got)) {
        if (et == 0) raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
        break;
      }
      tc::fence_after_sync();
      // paired: unit b of the pair fills rows 64 b .. of 128-row tiles
      unsigned char* B2 = sm + OFF_B2 + (PAIR ? sb * 8 * B_TILE + b * 64 * 128 : b * 4 * B_TILE);
      if (DT == 8) {
        constexpr int TS = PAIR ? 2 * B_TILE : B_TILE;           // tile stride
        unsigned char* bh = B2 + im * TS + nn * 128 + ((uu ^ nn) << 4);
#pragma unroll
        for (int c0 = cs; c0 < cs + 32; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 64 + c0), v);
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              __nv_bfloat16 h0, l0, h1, l1;
              split_bf16(v[8 * g + 2 * q], h0, l0);
              split_bf16(v[8 * g + 2 * q + 1], h1, l1);
              hw[q] = pack_bf16(h0, h1);
              lw[q] = pack_bf16(l0, l1);
            }
            unsigned char* dst = bh + ((c0 >> 3) + g) * 1024;    // row n' * 8 + n
            *reinterpret_cast<uint4*>(dst) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(dst + 2 * TS) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
      } else
#pragma unroll 1
      for (int c0 = cs; c0 < cs + 32; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 64 + c0), v);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int c = c0 + q;
          if (rv && c < D2) {
            const int np = c / D, up = c % D;
            const int brow = np * D + nn, kre = im * half + uu * D + up;
            const uint32_t off = swz(brow, kre & 63);
            __nv_bfloat16 h, l;
            split_bf16(v[q], h, l);
            *reinterpret_cast<__nv_bfloat16*>(B2 + (kre >> 6) * B_TILE + off) = h;
            *reinterpret_cast<__nv_bfloat16*>(B2 + (2 + (kre >> 6)) * B_TILE + off) = l;
          }
        }
      }
      fence_proxy_async();                       // generic writes -> tensor-core reads
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&c1_empty[b]);
      tc::bar_sync(1, EPI);
      if (et == 0 && last) tc::mbar_arrive(&b2_full[sb]);   // paired: both units are in
    }
  } else {
    // ---- epilogue 2: accumulator 2 (rows (ht,ht') Re / Im, columns
    // j = n' * D + n) -> rows (k,k',ht,ht') of the split T2 operand: hi at
    // column j (Re) or krpE/2 + j (Im), lo krpE further.  Each thread owns
    // one row and sixteen consecutive columns, i.e. two 16-byte chunks of hi
    // and two of lo; they go to a staging copy of the unit's output rows in
    // 64-column boxes with the 128-byte swizzle (32 lanes = 32 rows cover the
    // eight slots four times: conflict-free), and one thread stores the
    // boxes with TMA.  Accumulator columns j >= D^2 are exact zeros (zero
    // rows of the B operand), so a sixteen-column group that starts below
    // D^2 is staged whole; staging positions never written stay zero.
    const int et = tid - 64 - EPI, quarter = warp & 3, row = quarter * 32 + lane;
    const int cs = ((warp - 2 - EPI / 32) >> 2) * 32;
    const int r = row & 63, im = row >> 6;
    const bool rv = r < D2;
    const int half = a.krpE / 2, nbox = a.krpE / 32;
    unsigned char* stg = sm + OFF_STG + r * 128;
    const int hl = cs >> 5;                    // this warp copies E_top's hi (0) or lo (1) half
    int za = -1;                               // item whose E_top is in TMEM
    long long i = 0;
    int z = (int)(u0 / KK), kk = (int)(u0 % KK);
    for (long long u = u0; u < u1; ++u, ++i, kk = kk + 1 < KK ? kk + 1 : 0, z = kk ? z : z + 1) {
      if (z != za) {
        // first unit of an item: this thread's row of E_top (hi or lo half,
        // 128 bytes per 64-wide K chunk, read from global memory) becomes the
        // TMEM A operand of GEMM2.  Every GEMM2 of the previous item has
        // completed (this group consumed its last accumulator), so the TMEM
        // region is free.
        const uint4* erow = reinterpret_cast<const uint4*>(
            a.E + (size_t)z * (size_t)a.e_item + (size_t)row * (size_t)(2 * a.krpE) +
            (size_t)(hl * a.krpE));
        // one chunk in flight at a time: 32 words per thread (unrolling the
        // chunks would hold 64 and spill at the 96-register limit)
#pragma unroll 1
        for (int c = 0; c < a.nchunk; ++c) {
          uint32_t w[32];
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const uint4 v = __ldg(erow + c * 8 + g);
            w[4 * g] = v.x; w[4 * g + 1] = v.y; w[4 * g + 2] = v.z; w[4 * g + 3] = v.w;
          }
          tc::tmem_st32(tmem + ((uint32_t)(quarter * 32) << 16) + (hl ? TM_A2L : TM_A2H) +
                            (uint32_t)(c * 32), w);
        }
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(a2t_full);
        za = z;
      }
      // paired: accumulator b holds both units of pair i / 2, unit i % 2 in
      // columns 64 (i % 2) ..; it is waited for at the pair's first unit and
      // released after its second
      const int b = PAIR ? (int)((i >> 1) & 1) : (int)(i & 1);
      const long long ub = PAIR ? (i >> 2) : (i >> 1);
      const bool first = !PAIR || (i & 1) == 0, last = !PAIR || (i & 1) == 1;
      const uint32_t cbase = 128u + (uint32_t)(PAIR ? b * 128 + (int)(i & 1) * 64 : b * 64);
      bool got = true;
      if (et == 0) {
        if (first) got = tc::mbar_wait_sleep(&c2_full[b], (uint32_t)(ub & 1), T12_SLEEP_POLLS);
        tc::bulk_wait_read();                   // the staging block is free again
      }
      if (!tc::bar_and(2, EPI, got)) {
        if (et == 0) raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int c0 = cs; c0 < cs + 32; c0 += 16) {
        if (DT == 8 || c0 < D2) {                 // uniform over the warp
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + cbase + (uint32_t)c0, v);
          if (rv) {
            const int pos = im * half + c0;      // hi column of v[0]
            unsigned char* bx = stg + (pos >> 6) * STG_BOX;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                __nv_bfloat16 h0, l0, h1, l1;
                split_bf16(v[8 * g + 2 * q], h0, l0);
                split_bf16(v[8 * g + 2 * q + 1], h1, l1);
                hw[q] = pack_bf16(h0, h1);
                lw[q] = pack_bf16(l0, l1);
              }
              const int slot = ((((pos & 63) >> 3) + g) ^ (r & 7)) << 4;
              *reinterpret_cast<uint4*>(bx + slot) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(bx + (nbox / 2) * STG_BOX + slot) =
                  make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
          }
        }
      }
      if (last) {
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&c2_empty[b]);
      }
      fence_proxy_async();                       // staging writes -> TMA reads
      tc::bar_sync(2, EPI);
      if (et == 0) {
        for (int q = 0; q < nbox; ++q)
          tc::tma_store_3d(&mT2, sm + OFF_STG + q * STG_BOX, 64 * q, kk * D2, z);
        tc::bulk_commit();
      }
    }
    if (et == 0) tc::bulk_wait_all();           // every store has landed before exit
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, TM_COLS);
}

size_t t12_smem_bytes() { return T12_SMEM; }

cudaError_t t12_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_t12<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)T12_SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_t12<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T12_SMEM);
}

// Etop: the split top edge of this half (W.ETLd or W.ETRd, doubled A
// operand rows of 2 krpE BF16, rowsE rows per item), read by epilogue 2.
// The output (T2 split operand, W.T2s) is written through the plan's store
// map mapT2st, whose box is one unit's D^2 rows.
cudaError_t launch_t12(ntu_ctx* c, int n, const void* Etop) {
  const Plan& P = c->plan;
  T12Args a;
  a.D = P.D; a.K = P.K;
  a.nchunk = (int)(P.krpE / 64);
  a.krpY = (int)P.krpY; a.krpE = (int)P.krpE;
  a.k1 = (int)((2 * P.dp * P.D + 15) / 16);
  a.units = (long long)n * P.K * P.K;
  a.E = (const __nv_bfloat16*)Etop;
  a.e_item = P.rowsE * 2 * P.krpE;
  a.err = c->d_status;
  if (a.units == 0) return cudaSuccess;
  const int grid = (int)(a.units < c->sms ? a.units : c->sms);
  if (P.D == 8 && c->tune.t12_pair != 0)
    k_t12<8><<<grid, T12_THREADS, T12_SMEM, c->stream>>>(P.mapYs, P.mapQs, P.mapT2st, a);
  else
    k_t12<0><<<grid, T12_THREADS, T12_SMEM, c->stream>>>(P.mapYs, P.mapQs, P.mapT2st, a);
  return after_launch(c, "k_t12");
}

}  // namespace ntu
