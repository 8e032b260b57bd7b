// Tensor-core (tcgen05) GEMMs of the environment contraction (Fig. 4) for
// the NTU_MIXED_BF16X3 precision.
//
// A complex product C = A B^T is computed as one real GEMM: B keeps its
// interleaved (re, im) storage as a real K-major row of length 2K, and A is
// "doubled": complex row r becomes the real rows [Re, -Im, Re, -Im, ...] and
// [Im, Re, Im, Re, ...], placed 64 rows apart inside a 128-row tile, so that
// one 128 x N accumulator tile holds Re C in lanes 0-63 and Im C in lanes
// 64-127.  Each operand is stored split, x = hi + lo with hi = bf16(x) and
// lo = bf16(x - hi), as [hi | lo] halves of its row, and the kernel
// accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor memory.
//
// The kernel is persistent (one CTA per SM walks the 128 x 128 output tiles
// of all items) and warp-specialised: warp 0 fetches operands by TMA
// (128-byte swizzle) through a 4-stage mbarrier pipeline, warp 1 issues
// tcgen05.mma (M=128, N=128, K=16 per instruction) into one of two TMEM
// accumulators, and warps 2-17 drain the other accumulator: TMEM -> shared
// staging -> global stores through separable index tables, either as complex
// FP32 or directly as the split BF16 operand of the next GEMM.  The epilogue
// of one tile thus overlaps the loads and MMAs of the next.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "ntu_dev.cuh"
#include "ntu_impl.h"
#include "tc_sm103.cuh"

namespace ntu {

namespace {
constexpr int TBM = 128, TBN = 128, TBK = 64;
constexpr int TILE_A = TBM * TBK * 2, TILE_B = TBN * TBK * 2;
constexpr int EPI_WARPS = 16, TC_THREADS = 64 + 32 * EPI_WARPS;
constexpr int EPI_SLICES = EPI_WARPS / 4, SLICE_COLS = TBN / EPI_SLICES;  // column slices per TMEM quarter
static_assert((32 * EPI_WARPS) % TBN == 0, "epilogue threads per output column");
constexpr long long WAIT_LIMIT = 1ll << 28;
constexpr int SM_STAGE = TBN + 4;                 // staging pitch (floats), 16-byte rows
// The split-BF16 outputs (modes 1, 2) are written through a shared staging
// tile so that the 2-byte stores run along output rows; the FP32 output of
// the long-K join (mode 0) is written straight from registers and spends
// the space on two more pipeline stages instead.
template <int MODE> struct TcCfg {
  static constexpr int STAGES = MODE == 0 ? 6 : 4;
  static constexpr size_t STAGING = MODE == 0 ? 0 : (size_t)TBM * SM_STAGE * 4;
  static constexpr size_t SMEM = (size_t)STAGES * (TILE_A + TILE_B) + STAGING + 1024 + 1024;
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
};
}  // namespace

// MODE 0: complex FP32 output at out[rowC[m] + colC[n]].
// MODE 1: split B operand: row rowC[m] + colC[n], complex column
//         rowK[m] + colK[n] of a [rows][2 krp] BF16 array.
// MODE 2: split doubled A operand: as MODE 1 but complex row r goes to the
//         real rows (r/64)*128 + r%64 (Re part) and +64 (Im part).
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB,
                                                          TcArgs a, int items) {
  constexpr int TSTAGES = TcCfg<MODE>::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + TSTAGES * TILE_A;
  float* stage = (float*)(sB + TSTAGES * TILE_B);          // [128][SM_STAGE] (modes 1, 2)
  uint64_t* full = (uint64_t*)((unsigned char*)stage + TcCfg<MODE>::STAGING);
  uint64_t* empty = full + TSTAGES;
  uint64_t* accf = empty + TSTAGES;                        // [2] accumulator ready
  uint64_t* acce = accf + 2;                               // [2] accumulator drained
  uint64_t* done = acce + 2;                               // all MMAs retired
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  int* srow = (int*)(tmem_slot + 4);                      // [2][64] row offsets of a tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntN = (a.N + TBN - 1) / TBN;
  const int per_item = ntN * a.mtiles;
  const long long total = (long long)per_item * items;
  if (tid == 0) {
    for (int s = 0; s < TSTAGES; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { tc::mbar_init(&accf[b], 1); tc::mbar_init(&acce[b], EPI_WARPS); }
    tc::mbar_init(done, 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 2 * TBN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  // Per 64-wide K tile two stages: the hi halves of A and B, then the lo
  // halves; the three products hi*hi, hi*lo, lo*hi are issued once both
  // have landed, so every operand tile is fetched once.
  const int steps = 2 * a.kTiles;
  if (warp == 0) {
    if (lane == 0) {
      // ---- producer
      long long g = 0;
      int s = 0;                          // stage g % TSTAGES, phase (g / TSTAGES) & 1
      uint32_t ph = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const int z = (int)(t / per_item), rem = (int)(t % per_item);
        const int mt = rem / ntN, n0 = (rem % ntN) * TBN;
        for (int it = 0; it < steps; ++it, ++g, s = s + 1 < TSTAGES ? s + 1 : 0, ph ^= s ? 0u : 1u) {
          if (g >= TSTAGES && !tc::mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT)) {
            raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
            ok = false;
            break;
          }
          const int x = (it & 1) * a.krp + (it >> 1) * TBK;
          tc::mbar_expect_tx(&full[s], TILE_A + TILE_B);
          tc::tma_load_3d(sA + s * TILE_A, &tmA, &full[s], x, mt * TBM, z);
          tc::tma_load_3d(sB + s * TILE_B, &tmB, &full[s], x, n0, z);
        }
      }
      // no TMA copy may still be landing in shared memory when the CTA exits
      for (long long q = g - TSTAGES < 0 ? 0 : g - TSTAGES; q < g; ++q)
        if (!tc::mbar_wait(&full[q % TSTAGES], (uint32_t)((q / TSTAGES) & 1), WAIT_LIMIT))
          raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      const uint32_t idesc = tc::idesc_bf16_f32(TBM, TBN);
      int s = 0;                          // stage and phase of the next K stage
      uint32_t ph = 0;
      int i = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
        const int b = i & 1, ub = i >> 1;
        if (ub > 0 && !tc::mbar_wait(&acce[b], (uint32_t)((ub - 1) & 1), WAIT_LIMIT)) {
          raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(b * TBN);
        for (int it = 0; it < steps; it += 2) {
          const int sh = s;
          const uint32_t phh = ph;
          if (++s == TSTAGES) { s = 0; ph ^= 1u; }
          const int sl = s;
          const uint32_t phl = ph;
          if (++s == TSTAGES) { s = 0; ph ^= 1u; }
          if (!tc::mbar_wait(&full[sh], phh, WAIT_LIMIT) || !tc::mbar_wait(&full[sl], phl, WAIT_LIMIT)) {
            raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint64_t ah = tc::sdesc_k128(tc::smem_u32(sA + sh * TILE_A));
          const uint64_t bh = tc::sdesc_k128(tc::smem_u32(sB + sh * TILE_B));
          const uint64_t al = tc::sdesc_k128(tc::smem_u32(sA + sl * TILE_A));
          const uint64_t bl = tc::sdesc_k128(tc::smem_u32(sB + sl * TILE_B));
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            tc::mma_bf16(acc, ah + 2 * kk, bh + 2 * kk, idesc, (it | kk) != 0);
            tc::mma_bf16(acc, ah + 2 * kk, bl + 2 * kk, idesc, 1);
            tc::mma_bf16(acc, al + 2 * kk, bh + 2 * kk, idesc, 1);
          }
          tc::mma_commit(&empty[sh]);
          tc::mma_commit(&empty[sl]);
        }
        if (ok) tc::mma_commit(&accf[b]);
      }
      // every MMA issued has retired before TMEM is released
      tc::mma_commit(done);
      if (!tc::mbar_wait(done, 0, WAIT_LIMIT)) raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, columns
    // slice * SLICE_COLS .. + SLICE_COLS - 1 of the accumulator
    const int et = tid - 64, quarter = warp & 3, slice = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int ethreads = 32 * EPI_WARPS;
    int i = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      const int b = i & 1, ub = i >> 1;
      const bool got = tc::mbar_wait(&accf[b], (uint32_t)(ub & 1), WAIT_LIMIT);
      if (!tc::bar_and(1, ethreads, got)) {
        if (et == 0) raise_status(a.err, ST_TIMEOUT, WHY_TC_WAIT);
        break;
      }
      tc::fence_after_sync();
      const int z = (int)(t / per_item), rem = (int)(t % per_item);
      const int mt = rem / ntN, n0 = (rem % ntN) * TBN;
      if (MODE == 0) {
        // lane row < 64 holds Re, row >= 64 Im of complex row mt*64 + row % 64
        const int m = mt * 64 + (row & 63);
        float* o = (float*)a.out + 2 * (long long)z * a.sOut + (row >> 6);
#pragma unroll 1
        for (int c = slice * SLICE_COLS; c < (slice + 1) * SLICE_COLS; c += 16) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TBN + c), v);
          if (m < a.Mc) {
            const long long rb = a.rowC[m];
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (n0 + c + q < a.N) o[2 * (rb + a.colC[n0 + c + q])] = v[q];
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acce[b]);
        continue;
      }
#pragma unroll 1
      for (int c = slice * SLICE_COLS; c < (slice + 1) * SLICE_COLS; c += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TBN + c), v);
        float4* dst = reinterpret_cast<float4*>(stage + row * SM_STAGE + c);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[b]);          // accumulator b may be reused
      if (et < 64) {
        const int m = mt * 64 + et;
        srow[et] = m < a.Mc ? a.rowC[m] : 0;
        srow[64 + et] = m < a.Mc ? a.rowK[m] : 0;
      }
      tc::bar_sync(1, ethreads);                         // staging complete
      if (a.vec4) {
        // four consecutive columns per item: their (re, im) pairs are
        // consecutive in one output row (checked on the host), so hi and lo
        // each go out as one 16-byte store
        __nv_bfloat16* o = (__nv_bfloat16*)a.out + (long long)z * a.sOut;
        const int g4 = et % (TBN / 4);
        const int n = n0 + 4 * g4;
        if (n < a.N) {
          const long long cC = a.colC[n], cK = a.colK[n];
          for (int j = et / (TBN / 4); j < 64 && mt * 64 + j < a.Mc; j += ethreads / (TBN / 4)) {
            const float4 re = *reinterpret_cast<const float4*>(stage + j * SM_STAGE + 4 * g4);
            const float4 im = *reinterpret_cast<const float4*>(stage + (64 + j) * SM_STAGE + 4 * g4);
            store_split4(o, srow[j] + cC, srow[64 + j] + cK, a.pitch, a.krp_out, re, im,
                         MODE == 2);
          }
        }
      } else {
        // each thread keeps one output column; rows advance by ethreads / TBN
        const int nn = et % TBN, n = n0 + nn;
        if (n < a.N) {
          const long long cC = a.colC[n], cK = a.colK[n];
          __nv_bfloat16* o = (__nv_bfloat16*)a.out + (long long)z * a.sOut;
          for (int j = et / TBN; j < 64 && mt * 64 + j < a.Mc; j += ethreads / TBN) {
            const float re = stage[j * SM_STAGE + nn], im = stage[(64 + j) * SM_STAGE + nn];
            store_split(o, srow[j] + cC, srow[64 + j] + cK, a.pitch, a.krp_out, re, im,
                        MODE == 2);
          }
        }
      }
      tc::bar_sync(1, ethreads);                         // staging free again
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * TBN);
}

// --------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  return enc;
}

// 3-D map of a [items][rows][cols] BF16 array with 64 x 128 boxes and the
// 128-byte swizzle.  cols must be a multiple of 64 (so every row pitch and
// every box start are 16-byte aligned).
int tc_make_map(CUtensorMap* map, void* base, long long cols, long long rows, long long items,
                int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return NTU_EUNSUPPORTED;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)items};
  cuuint64_t strides[2] = {(cuuint64_t)cols * 2, (cuuint64_t)cols * rows * 2};
  cuuint32_t box[3] = {TBK, (cuuint32_t)box_rows, 1}, es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? NTU_OK : NTU_ECUDA;
}

cudaError_t tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcCfg<0>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcCfg<1>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcCfg<2>::SMEM);
  return e;
}

cudaError_t launch_tc_gemm(ntu_ctx* c, const TcOp& op, int n, void* out) {
  TcArgs a = op.args;
  const int* t = c->plan.d_tab;
  a.rowC = t + op.rowC; a.colC = t + op.colC;
  a.rowK = op.rowK >= 0 ? t + op.rowK : nullptr;
  a.colK = op.colK >= 0 ? t + op.colK : nullptr;
  a.out = out;
  a.err = c->d_status;
  a.mtiles = op.mtiles;
  const long long tiles = (long long)((a.N + TBN - 1) / TBN) * op.mtiles * n;
  const int grid = (int)(tiles < c->sms ? tiles : c->sms);
  if (grid <= 0) return cudaSuccess;
  if (op.mode == 0) {
    k_tc_gemm<0><<<grid, TC_THREADS, TcCfg<0>::SMEM, c->stream>>>(op.mapA, op.mapB, a, n);
  } else if (op.mode == 1) {
    k_tc_gemm<1><<<grid, TC_THREADS, TcCfg<1>::SMEM, c->stream>>>(op.mapA, op.mapB, a, n);
  } else {
    k_tc_gemm<2><<<grid, TC_THREADS, TcCfg<2>::SMEM, c->stream>>>(op.mapA, op.mapB, a, n);
  }
  return after_launch(c, "k_tc_gemm");
}

}  // namespace ntu
