// Gate split, gate application and QR reduction (Fig. 2(a,b)), recomposition
// of the updated site tensors (Fig. 2(e)), lattice orientation of the four
// bonds, single-site Trotter gates and the cluster estimator.
#include <cuda_runtime.h>

#include "ntu_dev.cuh"
#include "ntu_impl.h"

namespace ntu {

// ----------------------------------------------------------- gate split
// X[(sA', sA), (sB', sB)] = G[sA', sB', sA, sB] = U S V^H (Fig. 2(a)); for the
// first r singular triples G_A[:, k] = sqrt(s_k) u_k and
// G_B[:, k] = (u_k^H X) / sqrt(s_k); components with s_k <= 1e-15 s_1 are
// exact zeros.  With swap_sites the gate is read with its two sites
// exchanged, G'[x', y', x, y] = G[y', x', y, x], for bonds whose left-role site
// is B.  One CTA per item.
__global__ void __launch_bounds__(NTU_CTA) k_gate_split(int d, int r, int swap_sites,
                                                        const double2* __restrict__ G,
                                                        double2* __restrict__ GA,
                                                        double2* __restrict__ GB) {
  extern __shared__ __align__(16) unsigned char smem[];
  SvdSmem& S = *reinterpret_cast<SvdSmem*>(smem);
  double2* X = reinterpret_cast<double2*>(smem + sizeof(SvdSmem));   // 16 x 16
  const int item = blockIdx.x, tid = threadIdx.x;
  const int dd = d * d;
  const double2* g = G + (size_t)item * dd * dd;
  for (int idx = tid; idx < dd * dd; idx += NTU_CTA) {
    int row = idx / dd, col = idx % dd;
    int a1 = row / d, a0 = row % d, b1 = col / d, b0 = col % d;
    double2 v = swap_sites ? g[((b1 * d + a1) * d + b0) * d + a0]
                           : g[((a1 * d + b1) * d + a0) * d + b0];
    X[row * 16 + col] = v;
    S.A[col * 32 + row] = v;
  }
  __syncthreads();
  cta_svd_small(S, dd);
  double2* ga = GA + (size_t)item * dd * r;
  double2* gb = GB + (size_t)item * dd * r;
  const double s0 = S.s[0];
  for (int idx = tid; idx < dd * r; idx += NTU_CTA) {
    int a = idx / r, k = idx % r;
    bool keep = k < dd && S.s[k] > 1e-15 * s0 && s0 > 0.0;
    double2 va = cz(), vb = cz();
    if (keep) {
      double sk = S.s[k], rs = sqrt(sk);
      va = cscale(S.A[k * 32 + a], rs);
      double2 acc = cz();
      for (int i = 0; i < dd; ++i) acc = cfmac(S.A[k * 32 + i], X[i * 16 + a], acc);
      vb = cscale(acc, 1.0 / rs);
    }
    ga[idx] = va;
    gb[idx] = vb;
  }
}

// ---------------------------------------------------- gated site matrices
// Left role (side 0): M[(p', l, u, dn), (r_leg, k)] = sum_s GA[s', s, k] T[(s, c), l, u, r_leg, dn]
// Right role (side 1): M[(p', r, u, dn), (l_leg, k)] with GB.  Column-major.
__global__ void __launch_bounds__(NTU_CTA) k_gated(int d, int danc, int D, int r,
                                                   const double2* __restrict__ Ta,
                                                   const double2* __restrict__ Tb,
                                                   const double2* __restrict__ GA,
                                                   const double2* __restrict__ GB,
                                                   double2* __restrict__ Mg) {
  const int item = blockIdx.x, side = blockIdx.y;
  const int dp = d * danc, D2 = D * D, D3 = D2 * D, D4 = D3 * D;
  const int m = dp * D3, K = D * r;
  const double2* T = (side ? Tb : Ta) + (size_t)item * dp * D4;
  const double2* GX = (side ? GB : GA) + (size_t)item * d * d * r;
  double2* out = Mg + ((size_t)item * 2 + side) * m * K;
  for (int idx = blockIdx.z * NTU_CTA + threadIdx.x; idx < m * K; idx += NTU_CTA * gridDim.z) {
    int col = idx / m, row = idx % m;
    int leg = col / r, k = col % r;
    int n_ = row % D, t = row / D;
    int u = t % D; t /= D;
    int e = t % D; t /= D;
    int c = t % danc, tp = t / danc;
    int l = side ? leg : e, w = side ? e : leg;
    double2 acc = cz();
    for (int s = 0; s < d; ++s)
      acc = cfma(GX[(tp * d + s) * r + k],
                 T[(size_t)(s * danc + c) * D4 + l * D3 + u * D2 + w * D + n_], acc);
    out[(size_t)col * m + row] = acc;
  }
}

// ------------------------------------------- CholeskyQR2, double-FP32
// Thin QR of the column-major m x K gated matrix for the mixed contexts
// (Fig. 2(b)): G1 = M^H M = L1 L1^H, Q1 = M L1^{-H}; G2 = Q1^H Q1 = L2 L2^H,
// Q = Q1 L2^{-H}, R = L2^H L1^H.  Both Cholesky factors have a real positive
// diagonal, so R has one too and (Q, R) is the unique QR with that
// convention.  The m-long products (Gram matrices and Q) run in double-FP32
// arithmetic (FP32 issues at 64x the FP64 rate), the K x K factorisations and
// inverses in FP64.  The second pass restores orthogonality to working
// precision when kappa(M)^2 * 2^-48 << 1; the kernel flags the matrix for the
// Householder kernel instead when a factorisation fails or when
// min/max diag(L1) <= 1e-5.
struct QrDfSmem {
  double2 G[32 * 32];      // Gram matrix, then its Cholesky factor (column-major)
  double2 R1[32 * 32];     // L1^H (row-major, upper)
  double2 Ri[32 * 32];     // an upper-triangular inverse (row-major, FP64)
  float4 Rid[32 * 32];     // the same in double-FP32
  double red[2 * NTU_WARPS];
  int flag;
};

// G = X^H X (lower triangle, column-major, leading dimension K) from the
// column-major double-FP32 X (m x K); one warp per entry.
__device__ void qrdf_gram(const float4* __restrict__ X, int m, int K, double2* G) {
  const int wid = threadIdx.x >> 5, lid = threadIdx.x & 31;
  const int npair = K * (K + 1) / 2;
  for (int t = wid; t < npair; t += NTU_WARPS) {
    int c = 0, rem = t;                 // pair t -> (r >= c)
    while (rem >= K - c) { rem -= K - c; ++c; }
    const int r = c + rem;
    const float4* xr = X + (size_t)r * m;
    const float4* xc = X + (size_t)c * m;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = lid; i < m; i += 32) df_cmac<true>(acc, xr[i], xc[i]);
    acc = df_warp_sum(acc);
    if (lid == 0) G[(size_t)c * K + r] = df_join(acc);
  }
  __syncthreads();
}

// From the Cholesky factor L (column-major lower) of G: U = L^H into Ru
// (row-major), its inverse into Ri (FP64) and Rid (double-FP32).
__device__ void qrdf_factor_inverse(const double2* L, int K, double2* Ru, double2* Ri,
                                    float4* Rid) {
  const int tid = threadIdx.x;
  for (int idx = tid; idx < K * K; idx += NTU_CTA) {
    const int i = idx / K, j = idx % K;
    Ru[idx] = j >= i ? cconj(L[(size_t)i * K + j]) : cz();
  }
  __syncthreads();
  // column j of the inverse of the upper-triangular Ru, by back substitution
  for (int j = tid; j < K; j += NTU_CTA) {
    for (int i = K - 1; i >= 0; --i) {
      double2 v = cz();
      if (i <= j) {
        v = i == j ? make_double2(1.0, 0.0) : cz();
        for (int l = i + 1; l <= j; ++l) v = cfms(Ru[i * K + l], Ri[l * K + j], v);
        v = cscale(v, 1.0 / Ru[i * K + i].x);
      }
      Ri[i * K + j] = v;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < K * K; idx += NTU_CTA) Rid[idx] = df_split(Ri[idx]);
  __syncthreads();
}

// Row i of X R for the column-major m x K double-FP32 X and an upper
// triangular R (double-FP32, row-major K x K): out_j = sum_{l <= j} x_l
// R[l][j], the terms in ascending l.  The outputs are formed in chunks of
// four columns, highest first, each from one pass over the x_l it needs
// (a chunk of columns j reads x_l for l <= j only, so writing it in place
// leaves every x_l a lower chunk reads untouched); the row's entries come
// from L2 once per chunk instead of once per output.  JOIN: write the
// FP64 values to the row-major Q row instead of in place.
template <bool JOIN>
__device__ __forceinline__ void qrdf_row_times_upper(float4* X, int m, int K, int i,
                                                     const float4* Rd, double2* Qrow) {
  constexpr int CH = 4;                                 // columns per chunk (registers)
  for (int jc = (K - 1) / CH * CH; jc >= 0; jc -= CH) {
    float4 acc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int jend = jc + CH < K ? jc + CH : K;
    for (int l = 0; l < jend; ++l) {
      const float4 x = X[(size_t)l * m + i];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int j = jc + u;
        if (j < jend && l <= j) df_cmac<false>(acc[u], x, Rd[l * K + j]);
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int j = jc + u;
      if (j < jend) {
        if (JOIN) Qrow[j] = df_join(acc[u]);
        else X[(size_t)j * m + i] = acc[u];
      }
    }
  }
}

__global__ void __launch_bounds__(NTU_CTA) k_qr_df(int m, int K, const double2* __restrict__ Mg,
                                                   float4* __restrict__ Xg,
                                                   double2* __restrict__ QA, double2* __restrict__ RA,
                                                   double2* __restrict__ QB, double2* __restrict__ RB,
                                                   int* __restrict__ fallback, int* paths) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  QrDfSmem& S = *reinterpret_cast<QrDfSmem*>(qr_smem);
  const int item = blockIdx.x, side = blockIdx.y, tid = threadIdx.x;
  const size_t mk = (size_t)m * K;
  const double2* M = Mg + ((size_t)item * 2 + side) * mk;
  float4* X = Xg + ((size_t)item * 2 + side) * mk;
  // four independent loads per thread before the splits and stores (one
  // at a time left this loop latency-bound)
  for (size_t i0 = tid; i0 < mk; i0 += 4 * NTU_CTA) {
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t idx = i0 + (size_t)u * NTU_CTA;
      v[u] = idx < mk ? M[idx] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t idx = i0 + (size_t)u * NTU_CTA;
      if (idx < mk) X[idx] = df_split(v[u]);
    }
  }
  __syncthreads();
  // pass 1: G1 = M^H M = L1 L1^H, R1 = L1^H, Q1 = M R1^{-1} (in place)
  qrdf_gram(X, m, K, S.G);
  int ok = cta_cholesky(S.G, K, 0.0, &S.flag);
  if (ok) {
    double dmin = INFINITY, dmax = 0.0;
    for (int i = 0; i < K; ++i) {
      dmin = fmin(dmin, S.G[(size_t)i * K + i].x);
      dmax = fmax(dmax, S.G[(size_t)i * K + i].x);
    }
    ok = dmin > 1e-5 * dmax;
  }
  if (ok) {
    qrdf_factor_inverse(S.G, K, S.R1, S.Ri, S.Rid);
    // row i: q_j = sum_{l <= j} x_l Ri[l][j], in place
    for (int i = tid; i < m; i += NTU_CTA) qrdf_row_times_upper<false>(X, m, K, i, S.Rid, nullptr);
    __syncthreads();
    // pass 2: G2 = Q1^H Q1 = L2 L2^H, R2 = L2^H, Q = Q1 R2^{-1}, R = R2 R1
    qrdf_gram(X, m, K, S.G);
    ok = cta_cholesky(S.G, K, 0.0, &S.flag);
  }
  if (ok) {
    // R = L2^H R1 (upper) into S.Ri, written out before S.Ri is reused for
    // the inverse of L2^H
    double2* R2 = S.Ri;
    for (int idx = tid; idx < K * K; idx += NTU_CTA) {
      const int i = idx / K, j = idx % K;
      double2 acc = cz();
      for (int l = i; l <= j; ++l) acc = cfma(cconj(S.G[(size_t)i * K + l]), S.R1[l * K + j], acc);
      R2[idx] = acc;                     // (L2^H R1)[i][j], upper
    }
    __syncthreads();
    double2* Ro = (side ? RB : RA) + (size_t)item * K * K;
    for (int idx = tid; idx < K * K; idx += NTU_CTA) Ro[idx] = (idx % K) >= (idx / K) ? R2[idx] : cz();
    __syncthreads();
    qrdf_factor_inverse(S.G, K, S.R1, S.Ri, S.Rid);    // R1 <- L2^H, Ri / Rid <- its inverse
    double2* Qo = (side ? QB : QA) + (size_t)item * mk;
    for (int i = tid; i < m; i += NTU_CTA)
      qrdf_row_times_upper<true>(X, m, K, i, S.Rid, Qo + (size_t)i * K);
  }
  if (tid == 0) {
    fallback[item * 2 + side] = ok ? 0 : 1;
    if (ok && paths) atomicAdd(paths + 6, 1);
  }
}

size_t qr_df_smem_bytes() { return sizeof(QrDfSmem); }

// ------------------------------------------------------- Householder QR
// Thin QR of the column-major m x K gated matrix with R's diagonal made real
// non-negative (Fig. 2(b)).  Q is written row-major (m x K), R row-major
// (K x K).  One CTA per (item, side); with `only` set, only the matrices it
// flags (those the double-FP32 kernel left to this one).
__global__ void __launch_bounds__(NTU_CTA) k_qr(int m, int K, double2* __restrict__ Mg,
                                                double2* __restrict__ Qcm,
                                                double2* __restrict__ QA, double2* __restrict__ RA,
                                                double2* __restrict__ QB, double2* __restrict__ RB,
                                                const int* __restrict__ only, int* paths) {
  __shared__ double2 taus[32];
  __shared__ double betas[32];
  __shared__ double sred[2 * NTU_WARPS];
  const int item = blockIdx.x, side = blockIdx.y, tid = threadIdx.x;
  if (only && !only[item * 2 + side]) return;
  if (tid == 0 && paths) atomicAdd(paths + 7, 1);
  const int wid = tid >> 5, lid = tid & 31;
  double2* M = Mg + ((size_t)item * 2 + side) * m * K;
  double2* Qc = Qcm + ((size_t)item * 2 + side) * m * K;
  for (int j = 0; j < K; ++j) {
    double2* col = M + (size_t)j * m;
    Reflector R = cta_reflector(col + j, m - j, sred);
    __syncthreads();
    for (int i = j + 1 + tid; i < m; i += NTU_CTA) col[i] = cmul(col[i], R.scale);
    if (tid == 0) { taus[j] = R.tau; betas[j] = R.beta; col[j] = make_double2(1.0, 0.0); }
    __syncthreads();
    if (R.tau.x != 0.0 || R.tau.y != 0.0) {
      double2 ct = cconj(R.tau);
      for (int c = j + 1 + wid; c < K; c += NTU_WARPS) {
        double2* cc = M + (size_t)c * m;
        double2 dot = cz();
        for (int i = j + lid; i < m; i += 32) dot = cfmac(col[i], cc[i], dot);
        dot = warp_sum2(dot);
        double2 f = cmul(ct, dot);
        for (int i = j + lid; i < m; i += 32) cc[i] = cfms(f, col[i], cc[i]);
      }
      __syncthreads();
    }
  }
  // Q = H_0 ... H_{K-1} [I; 0]
  for (size_t idx = tid; idx < (size_t)m * K; idx += NTU_CTA)
    Qc[idx] = make_double2((idx % m) == (idx / m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int j = K - 1; j >= 0; --j) {
    double2 t = taus[j];
    if (t.x == 0.0 && t.y == 0.0) continue;
    const double2* v = M + (size_t)j * m;
    for (int c = j + wid; c < K; c += NTU_WARPS) {
      double2* qc = Qc + (size_t)c * m;
      double2 dot = cz();
      for (int i = j + lid; i < m; i += 32) dot = cfmac(v[i], qc[i], dot);
      dot = warp_sum2(dot);
      double2 f = cmul(t, dot);
      for (int i = j + lid; i < m; i += 32) qc[i] = cfms(f, v[i], qc[i]);
    }
    __syncthreads();
  }
  double2* Qo = (side ? QB : QA) + (size_t)item * m * K;
  double2* Ro = (side ? RB : RA) + (size_t)item * K * K;
  for (size_t idx = tid; idx < (size_t)m * K; idx += NTU_CTA) {
    int i = idx / K, c = idx % K;
    double sg = betas[c] < 0.0 ? -1.0 : 1.0;
    Qo[idx] = cscale(Qc[(size_t)c * m + i], sg);
  }
  for (int idx = tid; idx < K * K; idx += NTU_CTA) {
    int j = idx / K, c = idx % K;
    double sg = betas[j] < 0.0 ? -1.0 : 1.0;
    double2 v = c > j ? M[(size_t)c * m + j] : (c == j ? make_double2(betas[j], 0.0) : cz());
    Ro[idx] = cscale(v, sg);
  }
}

// ------------------------------------------------------------ recompose
// T' = Q M (Fig. 2(e)) put back into [p, l, u, r, dn] and normalised.
__global__ void __launch_bounds__(NTU_CTA) k_recompose(int dp, int D, int K,
                                                       const double2* __restrict__ QA,
                                                       const double2* __restrict__ QB,
                                                       const double2* __restrict__ MA,
                                                       const double2* __restrict__ MB,
                                                       double2* __restrict__ TaO,
                                                       double2* __restrict__ TbO, int df) {
  __shared__ double2 Ms[32 * 8];
  __shared__ float4 Mdf[32 * 8];
  __shared__ double sred[2 * NTU_WARPS];
  const int item = blockIdx.x, side = blockIdx.y, tid = threadIdx.x;
  const int D2 = D * D, D3 = D2 * D, D4 = D3 * D, m = dp * D3;
  const double2* Q = (side ? QB : QA) + (size_t)item * m * K;
  const double2* Mx = (side ? MB : MA) + (size_t)item * K * D;
  double2* out = (side ? TbO : TaO) + (size_t)item * dp * D4;
  for (int i = tid; i < K * D; i += NTU_CTA) { Ms[i] = Mx[i]; Mdf[i] = df_split(Mx[i]); }
  __syncthreads();
  double nrm2 = 0.0;
  if (df) {
    // mixed contexts: one row of Q per thread, split into FP32 pairs once and
    // multiplied in double-FP32 by all D columns of M (D <= 8)
    for (int row = tid; row < m; row += NTU_CTA) {
      float4 acc[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) acc[a] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k = 0; k < K; ++k) {
        const float4 q = df_split(Q[(size_t)row * K + k]);
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (a < D) df_cmac<false>(acc[a], q, Mdf[k * D + a]);
      }
      int n_ = row % D, t = row / D;
      int u = t % D; t /= D;
      int e = t % D; int p = t / D;
#pragma unroll
      for (int a = 0; a < 8; ++a)
        if (a < D) {
          const double2 v = df_join(acc[a]);
          const int l = side ? a : e, rr = side ? e : a;
          out[(size_t)p * D4 + l * D3 + u * D2 + rr * D + n_] = v;
          nrm2 += cabs2(v);
        }
    }
  } else
  for (int idx = tid; idx < m * D; idx += NTU_CTA) {
    int row = idx / D, a = idx % D;
    double2 acc = cz();
    for (int k = 0; k < K; ++k) acc = cfma(Q[(size_t)row * K + k], Ms[k * D + a], acc);
    int n_ = row % D, t = row / D;
    int u = t % D; t /= D;
    int e = t % D; int p = t / D;
    int l = side ? a : e, rr = side ? e : a;
    out[(size_t)p * D4 + l * D3 + u * D2 + rr * D + n_] = acc;
    nrm2 += cabs2(acc);
  }
  double nrm = sqrt(block_sum(nrm2, sred));
  double sc = nrm > 0.0 ? 1.0 / nrm : 1.0;
  __syncthreads();
  for (int idx = tid; idx < dp * D4; idx += NTU_CTA) out[idx] = cscale(out[idx], sc);
}

// ------------------------------------------------------------ orientation
// Bond b -> bond-0 orientation: bonds 1 and 3 rotate the lattice clockwise
// (new (l, u, r, dn) = old (dn, l, u, r)); bonds 2 and 3 put B in the left role.
__global__ void k_orient(int dp, int D, int bond, const double2* __restrict__ A,
                         const double2* __restrict__ B, double2* __restrict__ Ta,
                         double2* __restrict__ Tb) {
  const int D2 = D * D, D3 = D2 * D, D4 = D3 * D;
  const bool rot = (bond == 1 || bond == 3), swp = (bond >= 2);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < dp * D4; idx += gridDim.x * blockDim.x) {
    int i4 = idx % D, t = idx / D;
    int i3 = t % D; t /= D;
    int i2 = t % D; t /= D;
    int i1 = t % D; int p = t / D;
    int src = rot ? (p * D4 + i2 * D3 + i3 * D2 + i4 * D + i1) : idx;
    Ta[idx] = swp ? B[src] : A[src];
    Tb[idx] = swp ? A[src] : B[src];
  }
}

__global__ void k_deorient(int dp, int D, int bond, const double2* __restrict__ Ta,
                           const double2* __restrict__ Tb, double2* __restrict__ A,
                           double2* __restrict__ B) {
  const int D2 = D * D, D3 = D2 * D, D4 = D3 * D;
  const bool rot = (bond == 1 || bond == 3), swp = (bond >= 2);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < dp * D4; idx += gridDim.x * blockDim.x) {
    int i4 = idx % D, t = idx / D;
    int i3 = t % D; t /= D;
    int i2 = t % D; t /= D;
    int i1 = t % D; int p = t / D;
    int src = rot ? (p * D4 + i4 * D3 + i1 * D2 + i2 * D + i3) : idx;
    A[idx] = swp ? Tb[src] : Ta[src];
    B[idx] = swp ? Ta[src] : Tb[src];
  }
}

// ---------------------------------------------------- single-site gates
// T <- (O (x) 1_anc) T on the physical factor, then unit norm.  Block 0: A,
// block 1: B.
__global__ void __launch_bounds__(NTU_CTA) k_site_gate(int d, int danc, int D,
                                                       double2* __restrict__ A,
                                                       double2* __restrict__ B,
                                                       const double2* __restrict__ op) {
  __shared__ double2 O[16];
  __shared__ double sred[2 * NTU_WARPS];
  double2* T = blockIdx.x ? B : A;
  const int tid = threadIdx.x;
  const int D4 = D * D * D * D, dp = d * danc;
  if (tid < d * d) O[tid] = op[tid];
  __syncthreads();
  double nrm2 = 0.0;
  for (int idx = tid; idx < danc * D4; idx += NTU_CTA) {
    int c = idx / D4, rest = idx % D4;
    double2 in[4], o[4];
    for (int s = 0; s < d; ++s) in[s] = T[(size_t)(s * danc + c) * D4 + rest];
    for (int t = 0; t < d; ++t) {
      double2 acc = cz();
      for (int s = 0; s < d; ++s) acc = cfma(O[t * d + s], in[s], acc);
      o[t] = acc;
      nrm2 += cabs2(acc);
    }
    for (int t = 0; t < d; ++t) T[(size_t)(t * danc + c) * D4 + rest] = o[t];
  }
  double nrm = sqrt(block_sum(nrm2, sred));
  double sc = nrm > 0.0 ? 1.0 / nrm : 1.0;
  __syncthreads();
  for (int idx = tid; idx < dp * D4; idx += NTU_CTA) T[idx] = cscale(T[idx], sc);
}

// ------------------------------------------------------ cluster estimator
// <O> on site T with its four neighbours N closed by their leaf edge
// tensors, over the same network with the identity.  out[0] = num / den.
__global__ void __launch_bounds__(NTU_CTA) k_measure(int d, int danc, int D,
                                                     const double2* __restrict__ T,
                                                     const double2* __restrict__ N,
                                                     const double2* __restrict__ op,
                                                     double2* __restrict__ S1,
                                                     double2* __restrict__ S2,
                                                     double2* __restrict__ E,
                                                     double2* __restrict__ out) {
  __shared__ double sred[2 * NTU_WARPS];
  const int tid = threadIdx.x;
  const int dp = d * danc, D2 = D * D, D3 = D2 * D, D4 = D3 * D;
  // leaf edge tensors: El keeps r, Eu keeps dn, Er keeps l, Ed keeps u
  for (int idx = tid; idx < 4 * D2; idx += NTU_CTA) {
    int which = idx / D2, x = (idx % D2) / D, y = idx % D;
    double2 acc = cz();
    for (int p = 0; p < dp; ++p)
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b)
          for (int c = 0; c < D; ++c) {
            size_t ix, iy, base = (size_t)p * D4;
            if (which == 0) { ix = base + a * D3 + b * D2 + x * D + c; iy = base + a * D3 + b * D2 + y * D + c; }
            else if (which == 1) { ix = base + a * D3 + b * D2 + c * D + x; iy = base + a * D3 + b * D2 + c * D + y; }
            else if (which == 2) { ix = base + x * D3 + a * D2 + b * D + c; iy = base + y * D3 + a * D2 + b * D + c; }
            else { ix = base + a * D3 + x * D2 + b * D + c; iy = base + a * D3 + y * D2 + b * D + c; }
            acc = cfma(N[ix], cconj(N[iy]), acc);
          }
    E[idx] = acc;
  }
  __syncthreads();
  // contract the four legs of T one at a time: S <- sum_leg S * E_leg[leg, leg']
  const double2* src = T;
  double2* bufs[2] = {S1, S2};
  for (int leg = 0; leg < 4; ++leg) {
    double2* dst = bufs[leg & 1];
    const double2* El = E + leg * D2;      // leg 0: l uses El (keeps r), 1: u/Eu, 2: r/Er, 3: dn/Ed
    int stride = leg == 0 ? D3 : leg == 1 ? D2 : leg == 2 ? D : 1;
    for (int idx = tid; idx < dp * D4; idx += NTU_CTA) {
      int a = (idx / stride) % D;
      int base = idx - a * stride;
      double2 acc = cz();
      for (int x = 0; x < D; ++x) acc = cfma(src[base + x * stride], El[x * D + a], acc);
      dst[idx] = acc;
    }
    __syncthreads();
    src = dst;
  }
  // num = sum conj(T[q..]) O_full[q, p] V[p..]; den = sum conj(T[p..]) V[p..]
  double2 num = cz(), den = cz();
  for (int idx = tid; idx < dp * D4; idx += NTU_CTA) {
    int p = idx / D4, rest = idx % D4;
    int s = p / danc, c = p % danc;
    double2 v = src[idx];
    den = cfmac(T[idx], v, den);
    for (int t = 0; t < d; ++t) {
      double2 ov = cmul(op[t * d + s], v);
      num = cfmac(T[(size_t)(t * danc + c) * D4 + rest], ov, num);
    }
  }
  num = block_sum2(num, sred);
  den = block_sum2(den, sred);
  if (tid == 0) out[0] = cdiv(num, den);
}

// ------------------------------------------------------------ launchers
static size_t gate_split_smem() { return sizeof(SvdSmem) + 16 * 16 * sizeof(double2); }

cudaError_t gate_qr_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_gate_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gate_split_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_qr_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)qr_df_smem_bytes());
}

static inline int grid_for(long long work) {
  long long b = (work + NTU_CTA - 1) / NTU_CTA;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_gate_qr(ntu_ctx* c, int n, const double2* Ta, const double2* Tb,
                           const double2* G, int swap_sites, double2* QA, double2* RA,
                           double2* QB, double2* RB) {
  const Plan& P = c->plan;
  Work& W = c->w;
  const size_t sm = gate_split_smem();
  k_gate_split<<<n, NTU_CTA, sm, c->stream>>>(P.d, P.r, swap_sites, G, W.GA, W.GB);
  cudaError_t e = after_launch(c, "k_gate_split");
  if (e != cudaSuccess) return e;
  int zsplit = (P.m * P.K + NTU_CTA * 8 - 1) / (NTU_CTA * 8);
  if (zsplit < 1) zsplit = 1;
  k_gated<<<dim3(n, 2, zsplit), NTU_CTA, 0, c->stream>>>(P.d, P.d_anc, P.D, P.r, Ta, Tb, W.GA,
                                                         W.GB, W.Mg);
  e = after_launch(c, "k_gated");
  if (e != cudaSuccess) return e;
  if (c->cfg.precision != NTU_FP64) {
    const size_t sq = qr_df_smem_bytes();
    k_qr_df<<<dim3(n, 2), NTU_CTA, sq, c->stream>>>(P.m, P.K, W.Mg, (float4*)W.Qcm, QA, RA, QB,
                                                   RB, W.qrflag, c->d_paths);
    e = after_launch(c, "k_qr_df");
    if (e != cudaSuccess) return e;
    // Householder for the matrices the double-FP32 kernel handed back
    k_qr<<<dim3(n, 2), NTU_CTA, 0, c->stream>>>(P.m, P.K, W.Mg, W.Qcm, QA, RA, QB, RB, W.qrflag,
                                                 c->d_paths);
    return after_launch(c, "k_qr");
  }
  k_qr<<<dim3(n, 2), NTU_CTA, 0, c->stream>>>(P.m, P.K, W.Mg, W.Qcm, QA, RA, QB, RB, nullptr,
                                               c->d_paths);
  return after_launch(c, "k_qr");
}

cudaError_t launch_recompose(ntu_ctx* c, int n, const double2* QA, const double2* QB,
                             const double2* MA, const double2* MB, double2* Ta_out,
                             double2* Tb_out) {
  const Plan& P = c->plan;
  k_recompose<<<dim3(n, 2), NTU_CTA, 0, c->stream>>>(P.dp, P.D, P.K, QA, QB, MA, MB, Ta_out,
                                                     Tb_out, c->cfg.precision != NTU_FP64);
  return after_launch(c, "k_recompose");
}

cudaError_t launch_orient(ntu_ctx* c, int bond, const double2* A, const double2* B,
                          double2* Ta, double2* Tb) {
  const Plan& P = c->plan;
  k_orient<<<grid_for(P.szT), NTU_CTA, 0, c->stream>>>(P.dp, P.D, bond, A, B, Ta, Tb);
  return after_launch(c, "k_orient");
}

cudaError_t launch_deorient(ntu_ctx* c, int bond, const double2* Ta, const double2* Tb,
                            double2* A, double2* B) {
  const Plan& P = c->plan;
  k_deorient<<<grid_for(P.szT), NTU_CTA, 0, c->stream>>>(P.dp, P.D, bond, Ta, Tb, A, B);
  return after_launch(c, "k_deorient");
}

cudaError_t launch_site_gate(ntu_ctx* c, double2* A, double2* B, const double2* op) {
  const Plan& P = c->plan;
  k_site_gate<<<2, NTU_CTA, 0, c->stream>>>(P.d, P.d_anc, P.D, A, B, op);
  return after_launch(c, "k_site_gate");
}

cudaError_t launch_measure(ntu_ctx* c, const double2* T, const double2* N, const double2* op,
                           double2* out) {
  const Plan& P = c->plan;
  Work& W = c->w;
  k_measure<<<1, NTU_CTA, 0, c->stream>>>(P.d, P.d_anc, P.D, T, N, op, W.mscr1, W.mscr2,
                                          W.medge, out);
  return after_launch(c, "k_measure");
}

}  // namespace ntu
