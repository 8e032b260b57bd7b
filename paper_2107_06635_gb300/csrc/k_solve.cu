// FP64 solvers of the bond update: Hermitisation and non-negativity repair
// of the metric g (Sec. II), the slicing of g for the tensor-core build of
// the ALS reduced metric, and the host side of the ALS truncation of Fig. 5
// (argument set-up and the choice of instantiation; the kernel is in
// als_kernel.cuh).  One CTA per bond update.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "ntu_dev.cuh"
#include "ntu_impl.h"
#include "als_types.cuh"
#include "oz_build.cuh"

namespace ntu {

__device__ __forceinline__ double2 ld2(const double2* p) { return *p; }
__device__ __forceinline__ double2 ld2(const float2* p) {
  float2 v = *p;
  return make_double2((double)v.x, (double)v.y);
}

// ------------------------------------------------------------- repair
// g <- (g + g^H)/2.  g is positive definite, and clipping its negative
// eigenvalues would change nothing, when the Gershgorin discs of the rows
// lie right of zero (min_i d_i - s_i > 0, s_i = sum_{j != i} |Re| + |Im| >=
// sum_{j != i} |g_ij|) or, failing that, when a Cholesky factorisation of g
// succeeds; otherwise g = W diag(max(lambda, 0)) W^H from a full
// eigendecomposition.  Finally g /= trace(g).
// diag = [||g - g^H|| / ||g||, lambda_min / lambda_max (NaN on the two
// certified paths), log(trace)].
template <typename C2in>
__global__ void __launch_bounds__(NTU_CTA) k_repair(int ng, const C2in* __restrict__ graw,
                                                    double2* __restrict__ g,
                                                    double2* __restrict__ scr,
                                                    double2* __restrict__ Wv,
                                                    double* __restrict__ Z,
                                                    double* __restrict__ de,
                                                    double2* __restrict__ tau,
                                                    double2* __restrict__ pv,
                                                    double* __restrict__ diag, int* status,
                                                    int* paths) {
  extern __shared__ __align__(16) double chain[];   // 2 * ng (also n_g float4 for the Cholesky)
  __shared__ double sred[2 * NTU_WARPS];
  __shared__ int sh[4];
  __shared__ int okflag;
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
  const long long item = blockIdx.x;
  const size_t nn = (size_t)ng * ng;
  const C2in* gr = graw + item * nn;
  double2* gi = g + item * nn;
  double2* sc = scr + item * nn;
  // 1. Hermiticity defect, Gershgorin discs and trace of the Hermitian part,
  // one warp per row
  double n2 = 0.0, h2 = 0.0, glo = INFINITY, trw = 0.0;
  if (std::is_same<C2in, float2>::value) {
    // FP32 raw metric (mixed contexts): the statistics and the disc radii in
    // FP32 (relative rounding < 2e-5 for n_g <= 1024 terms, covered by
    // inflating the radii by 1e-4); the diagonal Re g_rr is exact
    const float2* gf = reinterpret_cast<const float2*>(gr);
    for (int r = wid; r < ng; r += NTU_WARPS) {
      float srf = 0.f, n2f = 0.f, h2f = 0.f;
      double dr = 0.0;
      for (int c = lid; c < ng; c += 32) {
        const float2 a = gf[(size_t)r * ng + c], b = gf[(size_t)c * ng + r];
        n2f = fmaf(a.x, a.x, fmaf(a.y, a.y, n2f));
        const float dx = a.x - b.x, dy = a.y + b.y;
        h2f = fmaf(dx, dx, fmaf(dy, dy, h2f));
        if (c == r) dr = (double)a.x;
        else srf += 0.5f * (fabsf(a.x + b.x) + fabsf(a.y - b.y));
      }
      n2 += (double)n2f;
      h2 += (double)h2f;
      srf = warp_sum_f(srf);
      dr = warp_sum(dr);                 // one lane holds the diagonal
      glo = fmin(glo, dr - (double)srf * (1.0 + 1e-4));
      trw += dr;
    }
  } else {
    for (int r = wid; r < ng; r += NTU_WARPS) {
      double sr = 0.0, dr = 0.0;
      for (int c = lid; c < ng; c += 32) {
        double2 a = ld2(gr + (size_t)r * ng + c), b = ld2(gr + (size_t)c * ng + r);
        double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        n2 += cabs2(a);
        h2 += cabs2(make_double2(a.x - b.x, a.y + b.y));
        if (c == r) dr = h.x;
        else sr += fabs(h.x) + fabs(h.y);
      }
      sr = warp_sum(sr);
      dr = warp_sum(dr);                 // one lane holds the diagonal
      glo = fmin(glo, dr - sr * (1.0 + 1e-12));   // margin for the rounding of s
      trw += dr;
    }
  }
  if (lid != 0) trw = 0.0;
  n2 = block_sum(n2, sred);
  h2 = block_sum(h2, sred);
  glo = block_min(glo, sred);
  const double trg = block_sum(trw, sred);
  const double herm = n2 > 0.0 ? sqrt(h2 / n2) : 0.0;
  if (glo > 0.0 && isfinite(glo) && trg > 0.0 && isfinite(trg)) {
    // certified by the discs: write (g + g^H) / (2 tr) directly
    // (a + conj b) / 2 is exact in FP64; scaling by inv / 2 rounds once
    const double hinv = 0.5 / trg;
    for (size_t idx = tid; idx < nn; idx += NTU_CTA) {
      int r = idx / ng, c = idx % ng;
      double2 a = ld2(gr + idx), b = ld2(gr + (size_t)c * ng + r);
      gi[idx] = make_double2((a.x + b.x) * hinv, (a.y - b.y) * hinv);
    }
    if (tid == 0) {
      if (paths) atomicAdd(paths + 3, 1);
      diag[item * 3 + 0] = herm;
      diag[item * 3 + 1] = __longlong_as_double(0x7ff8000000000000ULL);   // NaN
      diag[item * 3 + 2] = log(trg);
    }
    return;
  }
  // an FP32 raw metric (mixed contexts) is certified in double-FP32
  // arithmetic, which resolves it far below its own rounding; FP64 otherwise
  constexpr bool kDf = std::is_same<C2in, float2>::value;
  for (size_t idx = tid; idx < nn; idx += NTU_CTA) {
    int r = idx / ng, c = idx % ng;
    double2 a = ld2(gr + idx), b = ld2(gr + (size_t)c * ng + r);
    double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    gi[idx] = h;
    if (kDf) reinterpret_cast<float4*>(sc)[(size_t)c * ng + r] = df_split(h);
    else sc[(size_t)c * ng + r] = h;     // column-major copy
  }
  // 2. Cholesky of the lower triangle certifies positive definiteness
  __syncthreads();
  int ok = kDf ? cta_cholesky_df(reinterpret_cast<float4*>(sc), ng, &okflag,
                                 reinterpret_cast<float4*>(chain))
               : cta_cholesky(sc, ng, 0.0, &okflag);
  if (tid == 0 && paths) atomicAdd(paths + (ok ? 4 : 5), 1);
  double ratio = __longlong_as_double(0x7ff8000000000000ULL);   // NaN
  if (!ok) {
    // 3. full eigendecomposition and clipping of negative eigenvalues
    double2* ta = tau + item * ng;
    double2* pp = pv + item * ng;
    double* dd = de + item * 2 * ng;
    double* ee = dd + ng;
    double* Zi = Z + item * nn;
    double2* Wi = Wv + item * nn;
    for (size_t idx = tid; idx < nn; idx += NTU_CTA) {
      int r = idx / ng, c = idx % ng;
      sc[(size_t)c * ng + r] = gi[idx];
    }
    __syncthreads();
    cta_hetrd(sc, ng, dd, ee, ta, pp, sred);
    int st = cta_tridiag_qr_z(dd, ee, ng, Zi, chain, sh);
    if (st && tid == 0) raise_status(status, st, WHY_REPAIR_QR);
    // W = Q Z, one column per thread
    for (int k = tid; k < ng; k += NTU_CTA) {
      double2* col = Wi + (size_t)k * ng;
      for (int i = 0; i < ng; ++i) col[i] = make_double2(Zi[(size_t)i * ng + k], 0.0);
      for (int j = ng - 2; j >= 0; --j) {
        double2 t = ta[j];
        if (t.x == 0.0 && t.y == 0.0) continue;
        const double2* v = sc + (size_t)j * ng + j + 1;
        int m = ng - j - 1;
        double2 s = cz();
        for (int i = 0; i < m; ++i) s = cfmac(i == 0 ? make_double2(1.0, 0.0) : v[i], col[j + 1 + i], s);
        double2 f = cmul(t, s);
        for (int i = 0; i < m; ++i)
          col[j + 1 + i] = csub(col[j + 1 + i], cmul(f, i == 0 ? make_double2(1.0, 0.0) : v[i]));
      }
    }
    __syncthreads();
    double lmin = dd[0], lmax = dd[0];
    for (int i = 1; i < ng; ++i) { lmin = fmin(lmin, dd[i]); lmax = fmax(lmax, dd[i]); }
    ratio = lmax > 0.0 ? lmin / lmax : 0.0;
    for (size_t idx = tid; idx < nn; idx += NTU_CTA) {
      int r = idx / ng, c = idx % ng;
      double2 acc = cz();
      for (int k = 0; k < ng; ++k) {
        double lk = dd[k];
        if (lk <= 0.0) continue;
        acc = cfma(cscale(Wi[(size_t)k * ng + r], lk), cconj(Wi[(size_t)k * ng + c]), acc);
      }
      gi[idx] = acc;
    }
    __syncthreads();
  }
  // 4. unit trace
  double tr = 0.0;
  for (int i = tid; i < ng; i += NTU_CTA) tr += gi[(size_t)i * ng + i].x;
  tr = block_sum(tr, sred);
  if (!(tr > 0.0) || !isfinite(tr)) {
    if (tid == 0) raise_status(status, ST_NUMERIC, WHY_REPAIR_TRACE);
    tr = 1.0;
  }
  const double inv = 1.0 / tr;
  for (size_t idx = tid; idx < nn; idx += NTU_CTA) gi[idx] = cscale(gi[idx], inv);
  if (tid == 0) {
    diag[item * 3 + 0] = herm;
    diag[item * 3 + 1] = ratio;
    diag[item * 3 + 2] = log(tr);
  }
}

// ------------------------------------------- double-FP32 copy of g
// The mixed contexts' ALS reads g as double-FP32 pairs gdf = g 2^-e.  e = 0
// while max |Re|, |Im| lies in [2^-60, 2^60] (products and sums of the
// build then stay far inside the FP32 range); otherwise 2^e is the power of
// two just above the maximum, an exact scaling.  Two streaming passes over
// the batch, spread over every SM: the largest |Re|, |Im| of each item, then
// the split; for the lane build of the reduced metric also the copy
// gdfT[(kB',kA'),(kB,kA)] = gdf[(kA',kB'),(kA,kB)], which lets the B step
// read its blocks along rows as the A step does.  The maximum is taken on
// the bit patterns, whose order is that of the non-negative values; NaN
// entries are skipped.
__global__ void __launch_bounds__(NTU_CTA) k_gmax(long long nn, const double2* __restrict__ g,
                                                  unsigned long long* __restrict__ gmax) {
  __shared__ unsigned long long red[NTU_WARPS];
  const long long item = blockIdx.y;
  const double2* gi = g + item * nn;
  unsigned long long m = 0;
  for (long long i = blockIdx.x * (long long)NTU_CTA + threadIdx.x; i < nn;
       i += (long long)gridDim.x * NTU_CTA) {
    const double2 v = gi[i];
    unsigned long long a = dfb_bits(v.x) & 0x7fffffffffffffffull;
    unsigned long long b = dfb_bits(v.y) & 0x7fffffffffffffffull;
    if (a > 0x7ff0000000000000ull) a = 0;
    if (b > 0x7ff0000000000000ull) b = 0;
    m = max(m, max(a, b));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NTU_WARPS; ++w) m = max(m, red[w]);
    atomicMax(gmax + item, m);
  }
}

__device__ __forceinline__ int gscale_exp(unsigned long long mb) {
  const double mx = dfb_double(mb);
  return (mx > 0.0 && isfinite(mx) && (mx > 0x1p60 || mx < 0x1p-60)) ? ilogb(mx) + 1 : 0;
}

// Without the swapped copy a thread loads four entries of the item before
// it splits and stores them (one load at a time left the kernel latency-
// bound at a sixth of the HBM rate, measured); with it, one row of g per
// block iteration: row r of gdf is written in place, and row
// r' = (r mod K) K + r / K of gdfT, whose entry (c mod K) K + c / K is entry
// c of row r, from a copy staged in shared memory, so that both writes are
// contiguous, while the next row's entries are already being loaded.
constexpr int GSPLIT_BATCH = 4;
__global__ void __launch_bounds__(NTU_CTA) k_gsplit(int ng, int K, const double2* __restrict__ g,
                                                    const unsigned long long* __restrict__ gmax,
                                                    int* __restrict__ gscale,
                                                    float4* __restrict__ gdf,
                                                    float4* __restrict__ gdfT) {
  __shared__ float4 row[1024];                          // ng <= 1024
  const long long item = blockIdx.y, nn = (long long)ng * ng;
  const int e = gscale_exp(gmax[item]);
  if (blockIdx.x == 0 && threadIdx.x == 0) gscale[item] = e;
  const double2* gi = g + item * nn;
  float4* di = gdf + item * nn;
  if (!gdfT) {
    const long long step = (long long)gridDim.x * NTU_CTA;
    for (long long i0 = blockIdx.x * (long long)NTU_CTA + threadIdx.x; i0 < nn;
         i0 += GSPLIT_BATCH * step) {
      double2 v[GSPLIT_BATCH];
#pragma unroll
      for (int u = 0; u < GSPLIT_BATCH; ++u) {
        const long long i = i0 + u * step;
        v[u] = i < nn ? gi[i] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < GSPLIT_BATCH; ++u) {
        const long long i = i0 + u * step;
        if (i < nn) {
          if (e != 0) v[u] = make_double2(scalbn(v[u].x, -e), scalbn(v[u].y, -e));
          di[i] = df_split_bits(v[u]);
        }
      }
    }
    return;
  }
  float4* ti = gdfT + item * nn;
  constexpr int PER = 1024 / NTU_CTA;                   // entries of a row per thread, at most
  double2 cur[PER], nxt[PER];
  auto load_row = [&](int r, double2* dst) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int c = threadIdx.x + u * NTU_CTA;
      dst[u] = (r < ng && c < ng) ? gi[(size_t)r * ng + c] : make_double2(0.0, 0.0);
    }
  };
  load_row(blockIdx.x, cur);
  for (int r = blockIdx.x; r < ng; r += gridDim.x) {
    load_row(r + gridDim.x, nxt);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int c = threadIdx.x + u * NTU_CTA;
      if (c < ng) {
        double2 v = cur[u];
        if (e != 0) v = make_double2(scalbn(v.x, -e), scalbn(v.y, -e));
        const float4 d = df_split_bits(v);
        di[(size_t)r * ng + c] = d;
        row[(c % K) * K + c / K] = d;
      }
    }
    __syncthreads();
    float4* tr = ti + (size_t)((r % K) * K + r / K) * ng;
    for (int c = threadIdx.x; c < ng; c += NTU_CTA) tr[c] = row[c];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) cur[u] = nxt[u];
  }
}

size_t als_smem_bytes() { return sizeof(AlsShared); }

long long oz_rows_side(int K) { return oz_supported(K) ? oz_geo(K).rows_side : 0; }

cudaError_t launch_repair(ntu_ctx* c, int n, const void* graw, int raw_is_f32, double2* g,
                          double* diag) {
  const Plan& P = c->plan;
  Work& W = c->w;
  size_t sm = 2 * sizeof(double) * P.ng;
  if (raw_is_f32) {
    cudaFuncSetAttribute(k_repair<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_repair<float2><<<n, NTU_CTA, sm, c->stream>>>(P.ng, (const float2*)graw, g, W.gscr, W.gw,
                                                    W.gz, W.geig, W.gtau, W.gp, diag, c->d_status,
                                                    c->d_paths);
  } else {
    cudaFuncSetAttribute(k_repair<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_repair<double2><<<n, NTU_CTA, sm, c->stream>>>(P.ng, (const double2*)graw, g, W.gscr,
                                                     W.gw, W.gz, W.geig, W.gtau, W.gp, diag,
                                                     c->d_status, c->d_paths);
  }
  return after_launch(c, "k_repair");
}

cudaError_t launch_als(ntu_ctx* c, int n, const double2* g, const double2* RA,
                       const double2* RB, double2* MA, double2* MB, double* info, int sweeps) {
  const Plan& P = c->plan;
  Work& W = c->w;
  AlsArgs a;
  a.D = P.D; a.K = P.K; a.ng = P.ng; a.nA = P.nA;
  a.sweeps = sweeps < 0 ? c->cfg.als_sweeps : sweeps;
  a.kmin = c->cfg.tau_kmin; a.kmax = c->cfg.tau_kmax;
  a.g = g; a.RA = RA; a.RB = RB; a.MA = MA; a.MB = MB; a.info = info;
  a.x0 = W.x0; a.gx0 = W.gx0; a.Tm = W.Tm; a.gA = W.gA; a.gC = W.gC; a.jv = W.jv; a.pv = W.pv;
  a.path_counts = c->d_paths;
  a.tauv = W.tauv; a.dv = W.dv; a.ev = W.ev; a.rc = W.rc; a.rs = W.rs; a.rk = W.rk;
  a.rotcap = W.rotcap; a.status = c->d_status;
  a.df = c->cfg.precision != NTU_FP64;
  a.gdf = reinterpret_cast<float4*>(W.gscr);
  a.gdfT = reinterpret_cast<float4*>(W.gw);     // the repair's eigenvector scratch, free here
  size_t sm = sizeof(AlsShared);
  const int sms = c->sms;
  // a batch that leaves SMs idle gives each item 2 or 4 CTAs (one cluster),
  // as many as keep about one CTA per SM: co-resident CTAs of a cluster
  // mostly share the SM for the work they duplicate.  Measured on GB300:
  // at D = 8 up to one CTA per SM pays, at D <= 4 (a quarter of the solve
  // work per CTA) up to 1.5
  int split = a.df ? W.als_split : 1;
  const long long cap = P.D <= 4 ? 3LL * sms / 2 : (long long)sms;
  if (c->tune.als_split > 0) split = c->tune.als_split;   // ntu_set_tuning (<= W.als_split)
  else
    while (split > 1 && (long long)n * split > cap) split >>= 1;
  a.split = split;
  a.sync = W.als_sync;
  a.wait_polls = c->wait_polls;
  a.sync_extra = c->inject_timeout;
  // the tensor-core build of the reduced metric (K = 16 or 32, on one CTA
  // or a cluster) unless the tuning asks for the lane build.  Measured on
  // GB300 it takes 17-30 % off the ALS at K = 32 and up to 5 % at K = 16,
  // where a few cluster launches favour the lanes by as much
  a.oz = (c->plan.oz_ok && c->tune.als_build != 1) ? 1 : 0;
  a.gsl = reinterpret_cast<__nv_bfloat16*>(W.gsl);
  a.gexp = W.gexp;
  a.gmap = W.gmap;
  a.gscale = W.gscale;
  if (a.df) {
    // the double-FP32 copies of g, on every SM: blocks per item enough for
    // about eight per SM in all
    const long long nn = (long long)P.ng * P.ng;
    long long bx = (8LL * sms + n - 1) / n;
    const long long most = (nn + 4LL * NTU_CTA - 1) / (4LL * NTU_CTA);
    if (bx > most) bx = most;
    if (bx < 1) bx = 1;
    cudaError_t e = cudaMemsetAsync(W.gmaxb, 0, sizeof(unsigned long long) * (size_t)n, c->stream);
    if (e != cudaSuccess) return e;
    k_gmax<<<dim3((unsigned)bx, (unsigned)n), NTU_CTA, 0, c->stream>>>(nn, g, W.gmaxb);
    e = after_launch(c, "k_gmax");
    if (e != cudaSuccess) return e;
    long long bs = (8LL * sms + n - 1) / n;              // blocks per item
    if (bs > P.ng) bs = P.ng;
    k_gsplit<<<dim3((unsigned)bs, (unsigned)n), NTU_CTA, 0, c->stream>>>(
        P.ng, P.K, g, W.gmaxb, W.gscale, a.gdf, a.oz ? nullptr : a.gdfT);
    e = after_launch(c, "k_gsplit");
    if (e != cudaSuccess) return e;
  }
  if (a.oz) {
    // slices of every item's g for the tensor-core build
    const long long tasks = (long long)n * 2 * P.K * P.ng * (P.K / 4);
    long long blocks = (tasks + NTU_CTA - 1) / NTU_CTA;
    if (blocks > 16LL * sms) blocks = 16LL * sms;
    void (*sk)(int, const double2*, __nv_bfloat16*, short*) =
        P.K == 16 ? k_oz_slice<16> : k_oz_slice<32>;
    sk<<<(int)blocks, NTU_CTA, 0, c->stream>>>(n, g, reinterpret_cast<__nv_bfloat16*>(W.gsl),
                                               W.gexp);
    cudaError_t e = after_launch(c, "k_oz_slice");
    if (e != cudaSuccess) return e;
  }
  const size_t smk = sm + (a.oz ? ALS_OZ_SLACK : 0);
  if (split > 1) {
    cudaError_t e = cudaMemsetAsync(W.als_sync, 0, sizeof(int) * (size_t)n, c->stream);
    if (e != cudaSuccess) return e;
  }
  const bool three =
      split == 1 && (c->tune.als_ctas_per_sm ? c->tune.als_ctas_per_sm == 3 : n > 2 * sms);
  cudaError_t e = !a.oz ? als_launch_lanes(a, n, split, three, smk, c->stream)
                  : P.K == 16 ? als_launch_tc16(a, n, split, three, smk, c->stream)
                              : als_launch_tc32(a, n, split, three, smk, c->stream);
  if (e != cudaSuccess) return e;
  return after_launch(c, split > 1 ? (a.oz ? "k_als (cluster, tensor-core build)" : "k_als (cluster)")
                                   : (a.oz ? "k_als (tensor-core build)" : "k_als"));
}

}  // namespace ntu
