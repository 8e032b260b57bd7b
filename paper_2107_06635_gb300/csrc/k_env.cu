// Environment contraction of the eight-site neighbourhood (Fig. 4): edge
// double tensors (Fig. 4(a,b)), the two half networks with the double
// isometries (Fig. 4(c,d)) and their join into the metric g (Fig. 4(d,e)).
// Every step is one batched complex GEMM whose operands and result are
// addressed through separable index tables, so no permutation is ever
// materialised.  FP64 (double2) and FP32 (float2) instantiations.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ntu_dev.cuh"
#include "ntu_impl.h"

namespace ntu {

template <typename C2> struct CplxT;
template <> struct CplxT<double2> {
  typedef double R;
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static double2 mk(double a, double b) { return make_double2(a, b); }
};
template <> struct CplxT<float2> {
  typedef float R;
  __device__ static float2 zero() { return make_float2(0.f, 0.f); }
  __device__ static float2 mk(float a, float b) { return make_float2(a, b); }
};

struct GemmArgs {
  int M, N, Kd;
  const int* rowA; const int* kA; const int* kB; const int* colB; const int* rowC; const int* colC;
  int conjA, conjB;
  long long sA, sB, sC;
  const int* rowK; const int* colK;
  int mode, pitch, krp_out;
};

// Tile BM x BN per CTA, BK-deep k chunks, each thread TM x TN outputs.
template <typename C2, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_cgemm(GemmArgs g, const C2* __restrict__ A, const C2* __restrict__ B, C2* __restrict__ C) {
  typedef typename CplxT<C2>::R R;
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ C2 As[BK][BM];
  __shared__ C2 Bs[BK][BN];
  __shared__ int rA[BM], cB[BN], kAs[BK], kBs[BK];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long long b = blockIdx.z;
  const C2* Ab = A + b * g.sA;
  const C2* Bb = B + b * g.sB;
  C2* Cb = C + b * g.sC;
  for (int i = tid; i < BM; i += NT) rA[i] = (m0 + i < g.M) ? g.rowA[m0 + i] : -1;
  for (int i = tid; i < BN; i += NT) cB[i] = (n0 + i < g.N) ? g.colB[n0 + i] : -1;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  C2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = CplxT<C2>::zero();
  for (int k0 = 0; k0 < g.Kd; k0 += BK) {
    __syncthreads();
    for (int i = tid; i < BK; i += NT) {
      bool ok = k0 + i < g.Kd;
      kAs[i] = ok ? g.kA[k0 + i] : -1;
      kBs[i] = ok ? g.kB[k0 + i] : -1;
    }
    __syncthreads();
    for (int i = tid; i < BK * BM; i += NT) {
      int kk = i / BM, mm = i % BM;
      C2 v = CplxT<C2>::zero();
      if (rA[mm] >= 0 && kAs[kk] >= 0) {
        v = Ab[(long long)rA[mm] + kAs[kk]];
        if (g.conjA) v.y = -v.y;
      }
      As[kk][mm] = v;
    }
    for (int i = tid; i < BK * BN; i += NT) {
      int kk = i / BN, nn = i % BN;
      C2 v = CplxT<C2>::zero();
      if (cB[nn] >= 0 && kBs[kk] >= 0) {
        v = Bb[(long long)kBs[kk] + cB[nn]];
        if (g.conjB) v.y = -v.y;
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C2 a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          R re = acc[i][j].x, im = acc[i][j].y;
          re = fma(a[i].x, bb[j].x, re); re = fma(-a[i].y, bb[j].y, re);
          im = fma(a[i].x, bb[j].y, im); im = fma(a[i].y, bb[j].x, im);
          acc[i][j].x = re; acc[i][j].y = im;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int m = m0 + ty + i * (BM / TM);
    if (m >= g.M) continue;
    long long rc = g.rowC[m];
    if constexpr (sizeof(C2) == 8) {
      if (g.mode != 0) {      // split BF16 operand of a tensor-core GEMM
        __nv_bfloat16* ob = (__nv_bfloat16*)C + b * g.sC;
        const long long rk = g.rowK[m];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          int n = n0 + tx + j * (BN / TN);
          if (n >= g.N) continue;
          if (g.mode == 3)
            store_split_planar(ob, rc + g.colC[n], rk + g.colK[n], g.pitch, g.krp_out,
                               (float)acc[i][j].x, (float)acc[i][j].y);
          else
            store_split(ob, rc + g.colC[n], rk + g.colK[n], g.pitch, g.krp_out,
                        (float)acc[i][j].x, (float)acc[i][j].y, g.mode == 2);
        }
        continue;
      }
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int n = n0 + tx + j * (BN / TN);
      if (n < g.N) Cb[rc + g.colC[n]] = acc[i][j];
    }
  }
}

template <typename C2>
static cudaError_t run_gemm(ntu_ctx* c, const GemmOp& op, int n, const void* A, const void* B, void* C) {
  GemmArgs a;
  const int* t = c->plan.d_tab;
  a.M = op.M; a.N = op.N; a.Kd = op.Kd;
  a.rowA = t + op.rowA; a.kA = t + op.kA; a.kB = t + op.kB; a.colB = t + op.colB;
  a.rowC = t + op.rowC; a.colC = t + op.colC;
  a.conjA = op.conjA; a.conjB = op.conjB;
  a.sA = op.sA; a.sB = op.sB; a.sC = op.sC;
  a.mode = op.mode; a.pitch = op.pitch; a.krp_out = op.krp_out;
  a.rowK = op.mode ? t + op.rowK : nullptr;
  a.colK = op.mode ? t + op.colK : nullptr;
  constexpr int BM = 64, BN = 64, TM = 4, TN = 4;
  constexpr int BK = sizeof(C2) == 16 ? 8 : 16;
  dim3 grid((op.N + BN - 1) / BN, (op.M + BM - 1) / BM, n);
  k_cgemm<C2, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, c->stream>>>(
      a, (const C2*)A, (const C2*)B, (C2*)C);
  return after_launch(c, "k_cgemm");
}

// Gram matrix of one leg (the side edges E_L, E_R of Fig. 4(b)): for every
// item E[rowC[x] + colC[x']] = sum_k T[rowA[x] + kA[k]] conj(T[kA[k] + rowA[x']])
// with at most 64 pairs (x, x').  A 64 x 64 GEMM tile would leave almost every
// thread idle over the long contraction (dp D^3 terms); here thread (pair,
// group) sums every fourth term of one pair and the four groups are added in
// shared memory, one CTA per item.
template <typename C2>
__global__ void __launch_bounds__(256) k_gram(int D, int Kd, const int* __restrict__ rowA,
                                              const int* __restrict__ kA,
                                              const int* __restrict__ rowC,
                                              const int* __restrict__ colC, long long sT,
                                              long long sE, const C2* __restrict__ T,
                                              C2* __restrict__ E) {
  typedef typename CplxT<C2>::R R;
  __shared__ R red[2][4][64];
  const int tid = threadIdx.x, pr = tid & 63, grp = tid >> 6;
  const C2* Ti = T + (long long)blockIdx.x * sT;
  R re = 0, im = 0;
  if (pr < D * D) {
    const C2* tx = Ti + rowA[pr / D];
    const C2* ty = Ti + rowA[pr % D];
#pragma unroll 4
    for (int k = grp; k < Kd; k += 4) {
      const int o = kA[k];
      const C2 a = tx[o], b = ty[o];
      re = fma(a.x, b.x, fma(a.y, b.y, re));
      im = fma(a.y, b.x, fma(-a.x, b.y, im));
    }
  }
  red[0][grp][pr] = re;
  red[1][grp][pr] = im;
  __syncthreads();
  if (grp == 0 && pr < D * D) {
    const R sr = (red[0][0][pr] + red[0][1][pr]) + (red[0][2][pr] + red[0][3][pr]);
    const R si = (red[1][0][pr] + red[1][1][pr]) + (red[1][2][pr] + red[1][3][pr]);
    E[(long long)blockIdx.x * sE + rowC[pr / D] + colC[pr % D]] = CplxT<C2>::mk(sr, si);
  }
}

template <typename C2>
static cudaError_t run_gram(ntu_ctx* c, const GemmOp& op, int n, const void* T, void* E) {
  if (n == 0) return cudaSuccess;
  const int* t = c->plan.d_tab;
  k_gram<C2><<<n, 256, 0, c->stream>>>(op.M, op.Kd, t + op.rowA, t + op.kA, t + op.rowC,
                                       t + op.colC, op.sA, op.sC, (const C2*)T, (C2*)E);
  return after_launch(c, "k_gram");
}

// --------------------------------------------------------------- plan
// Table builder: composite index -> element offset, first listed factor
// slowest.  Each factor is (extent, stride).
struct TabBuilder {
  std::vector<int> tab;
  int add(std::initializer_list<std::pair<int, long long>> f) {
    int off = (int)tab.size();
    std::vector<std::pair<int, long long>> v(f);
    long long total = 1;
    for (auto& p : v) total *= p.first;
    for (long long i = 0; i < total; ++i) {
      long long rem = i, o = 0;
      for (int k = (int)v.size() - 1; k >= 0; --k) {
        long long idx = rem % v[k].first;
        rem /= v[k].first;
        o += idx * v[k].second;
      }
      tab.push_back((int)o);
    }
    return off;
  }
};

int plan_build(ntu_ctx* c) {
  Plan& P = c->plan;
  const ntu_config& cf = c->cfg;
  P.D = cf.D; P.d = cf.d_phys; P.d_anc = cf.d_anc; P.dp = P.d * P.d_anc; P.r = cf.r;
  const int D = P.D, dp = P.dp;
  P.K = D * P.r;
  const int K = P.K;
  P.m = dp * D * D * D;
  P.ng = K * K;
  P.nA = K * D;
  const long long D2 = D * D, D3 = D2 * D, D4 = D3 * D, K2 = (long long)K * K;
  P.szT = dp * D4; P.szQ = (long long)P.m * K; P.szR = K2; P.szE1 = D2; P.szE2 = D4;
  P.szS2 = D4 * K2; P.szG = K2 * K2;
  TabBuilder T;
  auto op = [&](int M, int N, int Kd, int rowA, int kA, int kB, int colB, int rowC, int colC,
                int cA, int cB, long long sA, long long sB, long long sC) {
    GemmOp o;
    memset(&o, 0, sizeof(o));
    o.M = M; o.N = N; o.Kd = Kd; o.rowA = rowA; o.kA = kA; o.kB = kB; o.colB = colB;
    o.rowC = rowC; o.colC = colC; o.conjA = cA; o.conjB = cB; o.sA = sA; o.sB = sB; o.sC = sC;
    o.mode = 0; o.rowK = o.colK = -1;
    return o;
  };
  // ---- edge double tensors, Gram form E = T^T conj(T) over the closed legs
  // E_L[x][x'] = sum_{p,l,u,n} Tb[p,l,u,x,n] conj(Tb[p,l,u,x',n])   (keeps r)
  {
    int rA = T.add({{D, D}});
    int kk = T.add({{dp, D4}, {D, D3}, {D, D2}, {D, 1}});
    int rC = T.add({{D, D}}), cC = T.add({{D, 1}});
    P.eL = op(D, D, dp * D3, rA, kk, kk, rA, rC, cC, 0, 1, P.szT, P.szT, D2);
  }
  // E_R[x][x'] = sum_{p,u,r,n} Ta[p,x,u,r,n] conj(...)   (keeps l)
  {
    int rA = T.add({{D, D3}});
    int kk = T.add({{dp, D4}, {D, D2}, {D, D}, {D, 1}});
    int rC = T.add({{D, D}}), cC = T.add({{D, 1}});
    P.eR = op(D, D, dp * D3, rA, kk, kk, rA, rC, cC, 0, 1, P.szT, P.szT, D2);
  }
  int rC4 = T.add({{D, D3}, {D, D2}});   // (x, y) -> (x*D + y) * D^2
  int cC4 = T.add({{D, D}, {D, 1}});     // (x', y') -> x'*D + y'
  // E_TL[x,y,x',y'] = sum_{p,l,u} Tb[p,l,u,x,y] conj(...)  (x = r, y = dn)
  {
    int rA = T.add({{D, D}, {D, 1}});
    int kk = T.add({{dp, D4}, {D, D3}, {D, D2}});
    P.eTL = op((int)D2, (int)D2, dp * (int)D2, rA, kk, kk, rA, rC4, cC4, 0, 1, P.szT, P.szT, D4);
  }
  // E_BL[x,y,x',y'] = sum_{p,l,n} Tb[p,l,y,x,n] conj(...)  (x = r, y = u)
  {
    int rA = T.add({{D, D}, {D, D2}});
    int kk = T.add({{dp, D4}, {D, D3}, {D, 1}});
    P.eBL = op((int)D2, (int)D2, dp * (int)D2, rA, kk, kk, rA, rC4, cC4, 0, 1, P.szT, P.szT, D4);
  }
  // E_TR[x,y,x',y'] = sum_{p,u,r} Ta[p,x,u,r,y] conj(...)  (x = l, y = dn)
  {
    int rA = T.add({{D, D3}, {D, 1}});
    int kk = T.add({{dp, D4}, {D, D2}, {D, D}});
    P.eTR = op((int)D2, (int)D2, dp * (int)D2, rA, kk, kk, rA, rC4, cC4, 0, 1, P.szT, P.szT, D4);
  }
  // E_BR[x,y,x',y'] = sum_{p,r,n} Ta[p,x,y,r,n] conj(...)  (x = l, y = u)
  {
    int rA = T.add({{D, D3}, {D, D2}});
    int kk = T.add({{dp, D4}, {D, D}, {D, 1}});
    P.eBR = op((int)D2, (int)D2, dp * (int)D2, rA, kk, kk, rA, rC4, cC4, 0, 1, P.szT, P.szT, D4);
  }
  // ---- half environment (Q rows (p, e, u, n), columns k)
  const long long DK = D * K, D2K = D2 * K, D3K = D3 * K, DK2 = D * K2, D2K2 = D2 * K2,
                  D3K2 = D3 * K2;
  // Y[p,e',u,n,k] = sum_e Q[p,e,u,n,k] E_side[e,e']
  {
    int rA = T.add({{dp, D3K}, {D, DK}, {D, K}, {K, 1}});
    int kA = T.add({{D, D2K}});
    int kB = T.add({{D, D}});
    int cB = T.add({{D, 1}});
    int cC = T.add({{D, D2K}});
    P.y = op(dp * (int)D2 * K, D, D, rA, kA, kB, cB, rA, cC, 0, 0, P.szQ, D2, P.szQ);
  }
  // T1[u,u',n,k,n',k'] = sum_{p,e'} Y[p,e',u,n,k] conj(Q[p,e',u',n',k'])
  {
    int rA = T.add({{D, DK}, {D, K}, {K, 1}});
    int kk = T.add({{dp, D3K}, {D, D2K}});
    int rC = T.add({{D, D3K2}, {D, DK2}, {K, DK}});
    int cC = T.add({{D, D2K2}, {D, K}, {K, 1}});
    P.t1 = op((int)D2K, (int)D2K, dp * D, rA, kk, kk, rA, rC, cC, 0, 1, P.szQ, P.szQ, P.szS2);
  }
  // T2[n,n',ht,ht',k,k'] = sum_{u,u'} E_top[ht,u,ht',u'] T1[u,u',n,k,n',k']
  {
    int rA = T.add({{D, D3}, {D, D}});
    int kA = T.add({{D, D2}, {D, 1}});
    int kB = T.add({{D, D3K2}, {D, D2K2}});
    int cB = T.add({{D, DK2}, {K, DK}, {D, K}, {K, 1}});
    int rC = T.add({{D, DK2}, {D, K2}});
    int cC = T.add({{D, D3K2}, {K, K}, {D, D2K2}, {K, 1}});
    P.t2 = op((int)D2, (int)D2K2, (int)D2, rA, kA, kB, cB, rC, cC, 0, 0, D4, P.szS2, P.szS2);
  }
  // H[hb,hb',ht,ht',k,k'] = sum_{n,n'} E_bot[hb,n,hb',n'] T2[n,n',ht,ht',k,k']
  {
    int rA = T.add({{D, D3}, {D, D}});
    int kA = T.add({{D, D2}, {D, 1}});
    int kB = T.add({{D, D3K2}, {D, D2K2}});
    int cB = T.add({{D, DK2}, {D, K2}, {K, K}, {K, 1}});
    int rC = T.add({{D, D3K2}, {D, D2K2}});
    P.h = op((int)D2, (int)D2K2, (int)D2, rA, kA, kB, cB, rC, cB, 0, 0, D4, P.szS2, P.szS2);
  }
  // g[(k',j'),(k,j)] = sum_h HL[h,k,k'] HR[h,j,j']
  {
    int rA = T.add({{K, K}, {K, 1}});
    int kk = T.add({{(int)D4, K2}});
    int rC = T.add({{K, K}, {K, (long long)K * K2}});
    int cC = T.add({{K, 1}, {K, K2}});
    P.join = op((int)K2, (int)K2, (int)D4, rA, kk, kk, rA, rC, cC, 0, 0, P.szS2, P.szS2, P.szG);
    // ---- split-BF16 tensor-core variant: geometry of the split operands
    auto up = [](long long x, long long q) { return (x + q - 1) / q * q; };
    P.krpE = up(2 * D2, 64);                    // real K of t2 / h: (u,u') or (n,n')
    P.krpJ = up(2 * D4, 64);                    // real K of the join: h
    P.rowsE = 128 * ((D2 + 63) / 64);           // doubled edge operands
    P.rowsT = up(D2 * K2, 128);                 // T1 / T2 as B operands
    P.rowsHL = 128 * ((K2 + 63) / 64);          // doubled H_L
    P.rowsHR = up(K2, 128);                     // H_R
    const int pE = (int)(2 * P.krpE), pJ = (int)(2 * P.krpJ);
    // edge tensors E[(x,y),(x',y')] as doubled A operands of t2 / h:
    // complex row (x, x'), complex column (y, y')
    int erC = T.add({{D, D}, {D, 0}}), ecC = T.add({{D, 1}, {D, 0}});
    int erK = T.add({{D, 0}, {D, D}}), ecK = T.add({{D, 0}, {D, 1}});
    auto as_split = [&](GemmOp o, int mode, long long sC, int pitch, int krp) {
      o.rowC = erC; o.colC = ecC; o.rowK = erK; o.colK = ecK;
      o.mode = mode; o.sC = sC; o.pitch = pitch; o.krp_out = krp;
      return o;
    };
    P.e2TL = as_split(P.eTL, 2, P.rowsE * pE, pE, (int)P.krpE);
    P.e2BL = as_split(P.eBL, 2, P.rowsE * pE, pE, (int)P.krpE);
    P.e2TR = as_split(P.eTR, 2, P.rowsE * pE, pE, (int)P.krpE);
    P.e2BR = as_split(P.eBR, 2, P.rowsE * pE, pE, (int)P.krpE);
    // the bottom edges are the A operands of h, whose B operand (T2 from
    // k_t12) has complex column (n', n) with Re and Im planar: K index
    // y' * D + y, mode 3; the top edges are the A operands of GEMM2 inside
    // k_t12, whose B operand has K (u, u') planar: mode 3, K order kept
    const int ebK = T.add({{D, 0}, {D, 1}}), ebKc = T.add({{D, 0}, {D, D}});
    for (GemmOp* o : {&P.e2BL, &P.e2BR}) {
      o->rowK = ebK; o->colK = ebKc; o->mode = 3;
    }
    P.e2TL.mode = 3;
    P.e2TR.mode = 3;
    // The composite column indices below are ordered so that each producer's
    // fastest column index is the consumer's K index: the split stores then
    // run along rows (coalesced) instead of across them.
    // Fused t1-t2 (k_t12.cu): Y as the doubled A operand with complex row
    // k*64 + u*D + n (64 rows per k, padding rows zero) and complex column
    // (p,e'); conj(Q) as the B operand with row k'*64 + n'*D + u' and column
    // (p,e') (both written by k_yq); the result goes to T2s, the B operand of
    // h: row (k,k',ht,ht'), complex column (n',n), Re at column c and Im at
    // krpE/2 + c of each half (planar).
    P.krpY = up(2LL * dp * D, 64);
    P.rowsY = 128LL * K;
    P.rowsQ = 64LL * K;
    // h: C[(hb,hb'),(k,k',ht,ht')] -> join operand: complex column
    // h = (hb,hb',ht,ht'); H_L doubled (A) with complex row (k,k'), H_R plain
    // (B) with row (k',k) so that the join writes g along its rows
    TcOp h;
    memset(&h, 0, sizeof(h));
    h.rowC = T.add({{D, 0}, {D, 0}});
    h.colC = T.add({{K, K}, {K, 1}, {D, 0}, {D, 0}});
    h.rowK = T.add({{D, D3}, {D, D2}});
    h.colK = T.add({{K, 0}, {K, 0}, {D, D}, {D, 1}});
    const int hcolR = T.add({{K, 1}, {K, K}, {D, 0}, {D, 0}});
    h.mtiles = (int)(P.rowsE / 128);
    h.args.kTiles = (int)(P.krpE / 64); h.args.krp = (int)P.krpE;
    h.args.Mc = (int)D2; h.args.N = (int)D2K2;
    h.args.pitch = pJ; h.args.krp_out = (int)P.krpJ;
    P.tc_hL = h;
    P.tc_hL.mode = 2; P.tc_hL.args.sOut = P.rowsHL * pJ;
    P.tc_hR = h;
    P.tc_hR.mode = 1; P.tc_hR.args.sOut = P.rowsHR * pJ; P.tc_hR.colC = hcolR;
    // join: g[(k',j'),(k,j)] = sum_h H_L[(k,k'),h] H_R[(j,j'),h], B rows (j',j)
    TcOp jn;
    memset(&jn, 0, sizeof(jn));
    jn.rowC = rC; jn.colC = T.add({{K, K2}, {K, 1}}); jn.rowK = -1; jn.colK = -1;
    jn.mode = 0;
    jn.mtiles = (int)(P.rowsHL / 128);
    jn.args.kTiles = (int)(P.krpJ / 64); jn.args.krp = (int)P.krpJ;
    jn.args.Mc = (int)K2; jn.args.N = (int)K2;
    jn.args.sOut = P.szG;
    P.tc_join = jn;
  }
  // Epilogue vectorisation of the split outputs: every aligned group of four
  // columns must land in one output row at four consecutive complex columns
  // starting at a multiple of four, for every row.
  auto vec4_ok = [&](const TcOp& o) {
    const std::vector<int>& t = T.tab;
    const int N = o.args.N, Mc = o.args.Mc;
    if (o.mode == 0 || N % 4 != 0) return 0;
    for (int m = 0; m < Mc; ++m)
      if (t[o.rowK + m] % 4 != 0) return 0;
    for (int n = 0; n < N; n += 4) {
      if (t[o.colK + n] % 4 != 0) return 0;
      for (int q = 1; q < 4; ++q)
        if (t[o.colC + n + q] != t[o.colC + n] || t[o.colK + n + q] != t[o.colK + n] + q) return 0;
    }
    return 1;
  };
  for (TcOp* o : {&P.tc_hL, &P.tc_hR, &P.tc_join})
    o->args.vec4 = vec4_ok(*o);
  P.n_tab = (int)T.tab.size();
  if (cudaMalloc(&P.d_tab, sizeof(int) * P.n_tab) != cudaSuccess) return NTU_ENOMEM;
  if (cudaMemcpy(P.d_tab, T.tab.data(), sizeof(int) * P.n_tab, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return NTU_ECUDA;
  return NTU_OK;
}

void plan_free(ntu_ctx* c) {
  if (c->plan.d_tab) cudaFree(c->plan.d_tab);
  c->plan.d_tab = nullptr;
}

// --------------------------------------------------------- conversions
__global__ void k_to_f32(long long n, const double2* __restrict__ in, float2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

static cudaError_t to_f32(ntu_ctx* c, long long n, const double2* in, void* out) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_to_f32<<<(int)blocks, 256, 0, c->stream>>>(n, in, (float2*)out);
  return after_launch(c, "k_to_f32");
}

__global__ void k_to_f64(long long n, const float2* __restrict__ in, double2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

cudaError_t launch_copy_raw(ntu_ctx* c, int n, const void* graw, double2* g) {
  long long cnt = (long long)n * c->plan.szG;
  long long blocks = (cnt + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_to_f64<<<(int)blocks, 256, 0, c->stream>>>(cnt, (const float2*)graw, g);
  return after_launch(c, "k_to_f64");
}

#define RG(x)                            \
  do {                                   \
    cudaError_t _e = (x);                \
    if (_e != cudaSuccess) return _e;    \
  } while (0)

template <typename C2>
static cudaError_t env_chain(ntu_ctx* c, int n, const void* Ta, const void* Tb, const void* QA,
                      const void* QB, void* graw) {
  const Plan& P = c->plan;
  Work& W = c->w;
  RG(run_gram<C2>(c, P.eL, n, Tb, W.EL));
  RG(run_gemm<C2>(c, P.eTL, n, Tb, Tb, W.ETL));
  RG(run_gemm<C2>(c, P.eBL, n, Tb, Tb, W.EBL));
  RG(run_gram<C2>(c, P.eR, n, Ta, W.ER));
  RG(run_gemm<C2>(c, P.eTR, n, Ta, Ta, W.ETR));
  RG(run_gemm<C2>(c, P.eBR, n, Ta, Ta, W.EBR));
  // left half: Q_A with E_L, E_TL, E_BL
  RG(run_gemm<C2>(c, P.y, n, QA, W.EL, W.Y));
  RG(run_gemm<C2>(c, P.t1, n, W.Y, QA, W.T1));
  RG(run_gemm<C2>(c, P.t2, n, W.ETL, W.T1, W.T2));
  RG(run_gemm<C2>(c, P.h, n, W.EBL, W.T2, W.HL));
  // right half: Q_B with E_R, E_TR, E_BR
  RG(run_gemm<C2>(c, P.y, n, QB, W.ER, W.Y));
  RG(run_gemm<C2>(c, P.t1, n, W.Y, QB, W.T1));
  RG(run_gemm<C2>(c, P.t2, n, W.ETR, W.T1, W.T2));
  RG(run_gemm<C2>(c, P.h, n, W.EBR, W.T2, W.HR));
  RG(run_gemm<C2>(c, P.join, n, W.HL, W.HR, graw));
  return cudaSuccess;
}

// Tensor maps of the split operands (the work space is fixed at init, so
// the maps are encoded once).
// The two operands of GEMM1 of the fused t1-t2 from one read of Q: thread
// (item, p, u, n, k) loads Q[p,e,u,n,k] for e < D and writes
//   Y[p,e',u,n,k] = sum_e Q[p,e,u,n,k] E_side[e][e']   (Fig. 4(c))
// as the doubled split A operand (complex row k*64 + u*D + n, column p*D + e')
// and conj(Q) as the split B operand (row k*64 + n*D + u, column p*D + e).
// The sum runs over e in order with the same FMA sequence as k_cgemm.
__global__ void __launch_bounds__(256) k_yq(long long total, int D, int K, const float2* __restrict__ Q,
                                            const float2* __restrict__ E, __nv_bfloat16* __restrict__ Ys,
                                            __nv_bfloat16* __restrict__ Qs, long long rows, long long szQ,
                                            long long sY, long long sQs, int pitch, int krp) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long item = i / rows;
    int rem = (int)(i % rows);
    const int k = rem % K; rem /= K;
    const int n = rem % D; rem /= D;
    const int u = rem % D;
    const int p = rem / D;
    const long long se = (long long)D * D * K;
    const float2* q = Q + item * szQ + (((long long)p * D * D + u) * D + n) * K + k;
    const float2* Ei = E + item * (long long)D * D;
    float2 qe[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) qe[e] = e < D ? q[e * se] : make_float2(0.f, 0.f);
    __nv_bfloat16* ys = Ys + item * sY;
    __nv_bfloat16* qs = Qs + item * sQs;
    const long long ry = (long long)k * 64 + u * D + n, rq = (long long)k * 64 + n * D + u;
    if (D == 8) {
      // the eight columns p*8 + e of a row are 32 contiguous bytes of each of
      // hi and lo: 16-byte stores (rows are pitch = 2 krp BF16 apart, p*8
      // complex columns are 32-byte aligned)
      uint32_t yrh[8], yrl[8], yih[8], yil[8], qh[8], ql[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int f = 0; f < 8; ++f) {
          const float2 a = qe[f], b = Ei[f * 8 + e];
          re = fmaf(a.x, b.x, re); re = fmaf(-a.y, b.y, re);
          im = fmaf(a.x, b.y, im); im = fmaf(a.y, b.x, im);
        }
        __nv_bfloat16 h0, l0, h1, l1, g0, m0, g1, m1;
        split_bf16(re, h0, l0);
        split_bf16(im, h1, l1);
        yrh[e] = pack_bf16(h0, __hneg(h1)); yrl[e] = pack_bf16(l0, __hneg(l1));
        yih[e] = pack_bf16(h1, h0);          yil[e] = pack_bf16(l1, l0);
        split_bf16(qe[e].x, g0, m0);
        split_bf16(-qe[e].y, g1, m1);
        qh[e] = pack_bf16(g0, g1); ql[e] = pack_bf16(m0, m1);
      }
      __nv_bfloat16* pr = ys + ((ry / 64) * 128 + ry % 64) * pitch + 2 * p * 8;
      __nv_bfloat16* pi = pr + 64LL * pitch;
      __nv_bfloat16* pq = qs + rq * pitch + 2 * p * 8;
      auto st2 = [](__nv_bfloat16* dst, const uint32_t* w) {
        reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
      };
      st2(pr, yrh); st2(pr + krp, yrl); st2(pi, yih); st2(pi + krp, yil);
      st2(pq, qh); st2(pq + krp, ql);
      continue;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (e >= D) break;
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        if (f >= D) break;
        const float2 a = qe[f], b = Ei[f * D + e];
        re = fmaf(a.x, b.x, re); re = fmaf(-a.y, b.y, re);
        im = fmaf(a.x, b.y, im); im = fmaf(a.y, b.x, im);
      }
      store_split(ys, ry, (long long)p * D + e, pitch, krp, re, im, 1);
      store_split(qs, rq, (long long)p * D + e, pitch, krp, qe[e].x, -qe[e].y, 0);
    }
  }
}

static cudaError_t launch_yq(ntu_ctx* c, int n, const float2* Q, const float2* E) {
  const Plan& P = c->plan;
  const long long rows = (long long)P.dp * P.D * P.D * P.K, total = (long long)n * rows;
  if (total == 0) return cudaSuccess;
  const long long want = (total + 255) / 256;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  k_yq<<<blocks, 256, 0, c->stream>>>(total, P.D, P.K, Q, E, (__nv_bfloat16*)c->w.Ys,
                                      (__nv_bfloat16*)c->w.Qs, rows, P.szQ,
                                      P.rowsY * 2 * P.krpY, P.rowsQ * 2 * P.krpY,
                                      (int)(2 * P.krpY), (int)P.krpY);
  return after_launch(c, "k_yq");
}

int tc_plan_maps(ntu_ctx* c) {
  Plan& P = c->plan;
  Work& W = c->w;
  const long long cap = W.cap, pE = 2 * P.krpE, pJ = 2 * P.krpJ;
  int st = NTU_OK;
  auto mk = [&](CUtensorMap* m, void* base, long long cols, long long rows) {
    if (st == NTU_OK) st = tc_make_map(m, base, cols, rows, cap);
  };
  mk(&P.mapYs, W.Ys, 2 * P.krpY, P.rowsY);
  if (st == NTU_OK) st = tc_make_map(&P.mapQs, W.Qs, 2 * P.krpY, P.rowsQ, cap, 64);
  mk(&P.tc_hL.mapA, W.EBLd, pE, P.rowsE);
  mk(&P.tc_hR.mapA, W.EBRd, pE, P.rowsE);
  mk(&P.tc_hL.mapB, W.T2s, pE, P.rowsT);
  if (st == NTU_OK) st = tc_make_map(&P.mapT2st, W.T2s, pE, P.rowsT, cap, (int)(P.D * P.D));
  P.tc_hR.mapB = P.tc_hL.mapB;
  mk(&P.tc_join.mapA, W.HLd, pJ, P.rowsHL);
  mk(&P.tc_join.mapB, W.HRs, pJ, P.rowsHR);
  return st;
}

// Environment with split-BF16 tensor-core products (Fig. 4): the small edge
// and Y products stay on the FP32 pipes; t1 writes its result as the B
// operand of t2, the edge tensors as the doubled A operands of t2 / h, and
// t2, h and the join run on tcgen05 (k_tc.cu).
static cudaError_t env_chain_bf16x3(ntu_ctx* c, int n, const void* Ta, const void* Tb,
                                    const void* QA, const void* QB, void* graw) {
  const Plan& P = c->plan;
  Work& W = c->w;
  RG(run_gram<float2>(c, P.eL, n, Tb, W.EL));
  RG(run_gram<float2>(c, P.eR, n, Ta, W.ER));
  RG(run_gemm<float2>(c, P.e2TL, n, Tb, Tb, W.ETLd));
  RG(run_gemm<float2>(c, P.e2BL, n, Tb, Tb, W.EBLd));
  RG(run_gemm<float2>(c, P.e2TR, n, Ta, Ta, W.ETRd));
  RG(run_gemm<float2>(c, P.e2BR, n, Ta, Ta, W.EBRd));
  RG(launch_yq(c, n, (const float2*)QA, (const float2*)W.EL));
  RG(launch_t12(c, n, W.ETLd));
  RG(launch_tc_gemm(c, P.tc_hL, n, W.HLd));
  RG(launch_yq(c, n, (const float2*)QB, (const float2*)W.ER));
  RG(launch_t12(c, n, W.ETRd));
  RG(launch_tc_gemm(c, P.tc_hR, n, W.HRs));
  RG(launch_tc_gemm(c, P.tc_join, n, graw));
  return cudaSuccess;
}

cudaError_t launch_env(ntu_ctx* c, int n, const double2* Ta, const double2* Tb,
                       const double2* QA, const double2* QB, void* graw) {
  const Plan& P = c->plan;
  Work& W = c->w;
  if (c->cfg.precision == NTU_FP64) return env_chain<double2>(c, n, Ta, Tb, QA, QB, graw);
  RG(to_f32(c, (long long)n * P.szT, Ta, W.Tac));
  RG(to_f32(c, (long long)n * P.szT, Tb, W.Tbc));
  RG(to_f32(c, (long long)n * P.szQ, QA, W.QAc));
  RG(to_f32(c, (long long)n * P.szQ, QB, W.QBc));
  if (c->cfg.precision == NTU_MIXED_BF16X3)
    return env_chain_bf16x3(c, n, W.Tac, W.Tbc, W.QAc, W.QBc, graw);
  return env_chain<float2>(c, n, W.Tac, W.Tbc, W.QAc, W.QBc, graw);
}

}  // namespace ntu
