// Device side of the ALS truncation of Fig. 5 / Eqs. 2-5 (SVDU start,
// tilting, reduced metric and source, pseudo-inverse with the tolerance that
// minimises eps, balancing) and the kernel template k_als.  Included by the
// translation units that instantiate it (k_als_lanes.cu, k_als_tc16.cu,
// k_als_tc32.cu), each compiled on its own so the instantiations build in
// parallel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <type_traits>

#include "als_types.cuh"

namespace ntu {

// ---------------------------------------------------------------- ALS
// Candidate relative tolerances 1e-k of the pseudo-inverse (Eq. 4), as
// correctly rounded decimal literals.
__device__ __forceinline__ double als_tau(int k) {
  switch (k) {
    case 0: return 1e0;   case 1: return 1e-1;  case 2: return 1e-2;  case 3: return 1e-3;
    case 4: return 1e-4;  case 5: return 1e-5;  case 6: return 1e-6;  case 7: return 1e-7;
    case 8: return 1e-8;  case 9: return 1e-9;  case 10: return 1e-10; case 11: return 1e-11;
    case 12: return 1e-12; case 13: return 1e-13; case 14: return 1e-14; case 15: return 1e-15;
    case 16: return 1e-16; case 17: return 1e-17; case 18: return 1e-18; case 19: return 1e-19;
    default: return 1e-20;
  }
}

// The double-FP32 split of the isometric factor (during a build) and of the
// CG direction (during a solve) live in the SVD work array W, which only the
// tilts use; this keeps the per-CTA footprint low enough for three CTAs per
// SM.
__device__ __forceinline__ float4* als_fdf(AlsShared& sm) { return reinterpret_cast<float4*>(sm.S.W); }
__device__ __forceinline__ float4* als_pdf(AlsShared& sm) { return reinterpret_cast<float4*>(sm.S.W) + 256; }


static __device__ void als_exchange(const AlsArgs& a, long long item, int& phase);

// out = g v in double-FP32 products from the split copy gdf = g 2^-ge (mixed
// contexts): v is split into the SVD array A (free outside the tilts); a
// warp takes two rows at a time, two accumulators per row and lane, and
// rescales by 2^ge.  When an item's ALS runs on `split` CTAs, CTA `rank`
// takes the rows rank, rank + split, ... and writes them into every CTA's
// copy of out (`cstride` elements apart, the first at out); the cluster
// then exchanges, so each copy holds all rows.
static __device__ void als_gmat_df(AlsShared& sm, const AlsArgs& a, const float4* gdf, int ge,
                                   const double2* v, double2* out, long long cstride, int ng,
                                   long long item, int rank, int split, int& phase) {
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
  float4* vdf = reinterpret_cast<float4*>(sm.S.A);           // ng <= 1024
  for (int i = tid; i < ng; i += NTU_CTA) vdf[i] = df_split(v[i]);
  __syncthreads();
  for (int r0 = rank + 2 * split * wid; r0 < ng; r0 += 2 * split * NTU_WARPS) {
    const int r1 = r0 + split;
    const bool two = r1 < ng;
    const float4* g0 = gdf + (size_t)r0 * ng;
    const float4* g1 = gdf + (size_t)(two ? r1 : r0) * ng;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a0 = z, a1 = z, b0 = z, b1 = z;
    for (int c = lid; c < ng; c += 64) {
      const float4 v0 = vdf[c];
      df_cmac<false>(a0, g0[c], v0);
      df_cmac<false>(b0, g1[c], v0);
      if (c + 32 < ng) {
        const float4 v1 = vdf[c + 32];
        df_cmac<false>(a1, g0[c + 32], v1);
        df_cmac<false>(b1, g1[c + 32], v1);
      }
    }
    df_add1(a0.x, a0.z, a1.x, a1.z);
    df_add1(a0.y, a0.w, a1.y, a1.w);
    df_add1(b0.x, b0.z, b1.x, b1.z);
    df_add1(b0.y, b0.w, b1.y, b1.w);
    a0 = df_warp_sum(a0);
    b0 = df_warp_sum(b0);
    if (lid == 0) {
      double2 y = df_join(a0), w = df_join(b0);
      if (ge != 0) {
        y = make_double2(scalbn(y.x, ge), scalbn(y.y, ge));
        w = make_double2(scalbn(w.x, ge), scalbn(w.y, ge));
      }
      for (int cp = 0; cp < split; ++cp) {
        out[cp * cstride + r0] = y;
        if (two) out[cp * cstride + r1] = w;
      }
    }
  }
  if (split > 1) als_exchange(a, item, phase);
  else __syncthreads();
}

// Rendezvous of the `split` CTAs of one item (one thread-block cluster, so
// they run at the same time): each adds one to the item's counter and waits
// until all have, for the phase-th time; global writes made before are then
// visible to all.  The wait is bounded: on running out it raises
// ST_TIMEOUT / WHY_ALS_SYNC and goes on (the results are then flagged).
static __device__ void als_exchange(const AlsArgs& a, long long item, int& phase) {
  __syncthreads();
  ++phase;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(a.sync + item, 1);
    const int target = phase * a.split + a.sync_extra;
    const volatile int* cnt = a.sync + item;
    long long it = 0;
    while (*cnt < target) {
      if (++it > a.wait_polls) {
        raise_status(a.status, ST_TIMEOUT, WHY_ALS_SYNC);
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
  }
  __syncthreads();
}

// Singular value decomposition of the K x K matrix X in sm.S.A (column q
// at A[q * 32], K <= 32) with the outputs of cta_svd_small: S.A = U, S.V = V
// (columns by descending singular value, phase convention), S.s.  The
// one-sided Jacobi SVD takes about eight sweeps on a general matrix but two
// or three on R^H when X P = Q R is a QR factorisation with the columns of
// X ordered by decreasing norm (R's rows are then graded); the SVD of X is
// U = Q V_R, V = P U_R from that of R^H = U_R S V_R^H.  The QR is K
// Householder steps: warp 0 forms the reflector, a warp per column applies
// it, and each thread updates its row of Q.  A nearly rank-deficient R
// (min |R_kk| <= 1e-10 max |R_kk|) takes the plain Jacobi SVD of X instead.
static __device__ void als_svd_square(AlsShared& sm, int K) {
  SvdSmem& S = sm.S;
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
  double2* X0 = S.W;                                   // the input, for the fallback
  double2* Q = sm.y;                                   // y, y2, p, ap: column q at q * 32
  double2* v0 = sm.MA;                                 // v_k of reflector k
  double2* beta = sm.MA + 32;                          // R_kk
  double* cf = reinterpret_cast<double*>(sm.MA + 64);  // 2 / |v|^2
  double* rk = cf + 32;                                // |R_kk|
  int* perm = reinterpret_cast<int*>(sm.MB);
  for (int j = wid; j < K; j += NTU_WARPS) {
    double a2 = lid < K ? cabs2(S.A[j * 32 + lid]) : 0.0;
    a2 = warp_sum(a2);
    if (lid == 0) S.s[j] = isfinite(a2) ? a2 : -1.0;
  }
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) X0[idx] = S.A[idx];
  __syncthreads();
  if (tid < K) {                                       // rank of column tid by norm, ties by index
    const double v = S.s[tid];
    int rank = 0;
    for (int j = 0; j < K; ++j) rank += (S.s[j] > v) || (S.s[j] == v && j < tid);
    perm[rank] = tid;
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) {
    const int i = idx & 31, k = idx >> 5;
    S.A[idx] = (k < K && i < K) ? X0[perm[k] * 32 + i] : cz();
    Q[idx] = make_double2(i == k && k < K ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    // H = I - c v v^H, v = x - beta e_k, beta = -e^{i arg alpha} |x| for the
    // rows k.. of column k: H x = beta e_k, |v|^2 = 2 |x| (|x| + |alpha|)
    if (wid == 0) {
      const double2 x = (lid >= k && lid < K) ? S.A[k * 32 + lid] : cz();
      const double nx = sqrt(warp_sum(cabs2(x)));
      const double2 al = S.A[k * 32 + k];
      const double aa = sqrt(cabs2(al));
      const double2 ph = aa > 0.0 ? make_double2(al.x / aa, al.y / aa) : make_double2(1.0, 0.0);
      if (lid == 0) {
        v0[k] = cscale(ph, aa + nx);
        beta[k] = cscale(ph, -nx);
        cf[k] = nx > 0.0 ? 1.0 / (nx * (nx + aa)) : 0.0;
        rk[k] = nx;
      }
    }
    __syncthreads();
    const double2 vk = v0[k];
    const double c = cf[k];
    for (int j = k + 1 + wid; j < K; j += NTU_WARPS) {   // a_j <- a_j - v (c v^H a_j)
      const double2 vi = lid == k ? vk : ((lid > k && lid < K) ? S.A[k * 32 + lid] : cz());
      const double2 aij = (lid >= k && lid < K) ? S.A[j * 32 + lid] : cz();
      const double2 w = cscale(warp_sum2(cmulc(vi, aij)), c);
      if (lid >= k && lid < K) S.A[j * 32 + lid] = cfms(vi, w, aij);
    }
    if (tid < K) {                                     // row tid of Q <- Q H
      double2 sa = cz();
      for (int l = k; l < K; ++l) sa = cfma(Q[l * 32 + tid], l == k ? vk : S.A[k * 32 + l], sa);
      sa = cscale(sa, c);
      for (int l = k; l < K; ++l)
        Q[l * 32 + tid] = cfms(sa, cconj(l == k ? vk : S.A[k * 32 + l]), Q[l * 32 + tid]);
    }
    __syncthreads();
    if (tid < K && tid >= k) S.A[k * 32 + tid] = tid == k ? beta[k] : cz();
    __syncthreads();
  }
  double lo = rk[0], hi = rk[0];
  for (int k = 1; k < K; ++k) {
    lo = rk[k] < lo ? rk[k] : lo;
    hi = rk[k] > hi ? rk[k] : hi;
  }
  if (!(lo > 1e-10 * hi) || !isfinite(hi)) {
    for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) S.A[idx] = X0[idx];
    __syncthreads();
    cta_svd_small(S, K);
    return;
  }
  // M = R^H (lower triangular) through V, then its SVD
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) {
    const int i = idx & 31, j = idx >> 5;             // M[i][j] = conj(R[j][i])
    S.V[idx] = (i < K && j < K && j <= i) ? cconj(S.A[i * 32 + j]) : cz();
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) S.A[idx] = S.V[idx];
  __syncthreads();
  cta_svd_cols(S, K, K, 0);
  // U = Q V_R into W; V = P U_R into V; U into A
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) {
    const int i = idx & 31, q = idx >> 5;
    double2 acc = cz();
    if (i < K && q < K)
      for (int l = 0; l < K; ++l) acc = cfma(Q[l * 32 + i], S.V[q * 32 + l], acc);
    S.W[idx] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) {
    const int k = idx & 31, q = idx >> 5;
    if (k < K && q < K) S.V[q * 32 + perm[k]] = S.A[q * 32 + k];
    else if (q >= K || k >= K) S.V[idx] = cz();
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) S.A[idx] = S.W[idx];
  __syncthreads();
  cta_svd_phase(S, K, K);
}

// X = MA MB^T -> SVD -> (MA, MB) by mode: 0 tilt before the A step
// (U S, conj(V)), 1 tilt before the B step (U, conj(V) S), 2 balance
// (U sqrt(S), conj(V) sqrt(S)).  With from_x0 the SVD input is X0 instead.
static __device__ void als_tilt(AlsShared& sm, const AlsArgs& a, int mode, const double2* X0) {
  const int tid = threadIdx.x, K = a.K, D = a.D;
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) {
    int i = idx & 31, j = idx >> 5;
    double2 v = cz();
    if (i < K && j < K) {
      if (X0) v = X0[i * K + j];
      else
        for (int q = 0; q < D; ++q) v = cfma(sm.MA[i * D + q], sm.MB[j * D + q], v);
    }
    sm.S.A[j * 32 + i] = v;
  }
  __syncthreads();
  // the preconditioned SVD pays from K = 24 on (measured on GB300: 4% off
  // the K = 32 ALS, 1% slower at K = 16, where the QR costs what it saves)
  if (K >= 24) als_svd_square(sm, K);
  else cta_svd_small(sm.S, K);
  if (tid == 0 && sm.S.bad) sm.err |= WHY_SVD_NONFINITE;
  for (int idx = tid; idx < K * D; idx += NTU_CTA) {
    int i = idx / D, q = idx % D;
    double2 u = cz(), vb = cz();
    double sv = 0.0;
    if (q < K) { u = sm.S.A[q * 32 + i]; vb = cconj(sm.S.V[q * 32 + i]); sv = sm.S.s[q]; }
    if (mode == 0) { sm.MA[idx] = cscale(u, sv); sm.MB[idx] = vb; }
    else if (mode == 1) { sm.MA[idx] = u; sm.MB[idx] = cscale(vb, sv); }
    else { double rs = sqrt(sv); sm.MA[idx] = cscale(u, rs); sm.MB[idx] = cscale(vb, rs); }
  }
  __syncthreads();
}

// Tilt (modes 0, 1) or balance (mode 2) from the factors of the previous
// half step without forming X = MA MB^T.  One factor is an isometry left by
// the previous SVD, the other (Y) came out of the last solve.  Mode 1: Y = MA
// and MB = conj(V), so X = Y V^H; with Y = P S Q^H, U = P and V' = V Q, hence
// MA = P and MB = MB conj(Q) S.  Modes 0 and 2: Y = MB and MA = U, so
// X = MA conj(Q) S P^T, U' = MA conj(Q) and V' = conj(P), hence MA = U' S and
// MB = P (mode 0), or MA = U' sqrt(S) and MB = P sqrt(S) (mode 2).  U' gets
// the phase convention of the square SVD, V' the same phases.  The thin SVD
// of the K x D factor replaces the SVD of the K x K product of rank D.
// Returns 0 with MA and MB untouched when Y is numerically rank deficient
// (s_min <= 1e-14 s_max): the null directions of X then come from the square
// SVD of als_tilt.
static __device__ int als_tilt_fast(AlsShared& sm, const AlsArgs& a, int mode) {
  const int tid = threadIdx.x, K = a.K, D = a.D;
  const double2* Y = mode == 1 ? sm.MA : sm.MB;
  const double2* Z = mode == 1 ? sm.MB : sm.MA;
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) {
    int i = idx & 31, q = idx >> 5;
    sm.S.A[idx] = (i < K && q < D) ? Y[i * D + q] : cz();
  }
  __syncthreads();
  cta_svd_cols(sm.S, K, D, mode == 1);
  if (sm.S.bad || !(sm.S.s[D - 1] > 1e-14 * sm.S.s[0])) return 0;
  // W = Z conj(Q), K x D column-major
  for (int idx = tid; idx < 32 * 32; idx += NTU_CTA) {
    int i = idx & 31, q = idx >> 5;
    double2 acc = cz();
    if (i < K && q < D)
      for (int p = 0; p < D; ++p) acc = cfma(Z[i * D + p], cconj(sm.S.V[q * 32 + p]), acc);
    sm.S.W[idx] = acc;
  }
  __syncthreads();
  if (mode == 1) {
    for (int idx = tid; idx < K * D; idx += NTU_CTA) {
      int i = idx / D, q = idx % D;
      sm.MA[idx] = sm.S.A[q * 32 + i];
      sm.MB[idx] = cscale(sm.S.W[q * 32 + i], sm.S.s[q]);
    }
    __syncthreads();
    return 1;
  }
  // phase of each column of U' = W: its first entry within 1e-10 of the
  // largest modulus becomes real positive
  const int grp = tid >> 4, lane = tid & 15;
  const unsigned mask = 0xffffu << (tid & 16);
  for (int k = grp; k < D; k += 16) {
    double mx = 0.0;
    for (int r = lane; r < K; r += 16) mx = fmax(mx, cabs2(sm.S.W[k * 32 + r]));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(mask, mx, o));
    mx = sqrt(mx);
    int piv = 1 << 30;
    for (int r = lane; r < K; r += 16)
      if (mx > 0.0 && sqrt(cabs2(sm.S.W[k * 32 + r])) >= (1.0 - 1e-10) * mx) piv = min(piv, r);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) piv = min(piv, __shfl_xor_sync(mask, piv, o));
    double2 ph = make_double2(1.0, 0.0);
    if (mx > 0.0 && isfinite(mx) && piv < K) {
      double2 up = sm.S.W[k * 32 + piv];
      double am = sqrt(cabs2(up));
      ph = make_double2(up.x / am, -up.y / am);
    }
    if (lane == 0) sm.ph[k] = ph;
  }
  __syncthreads();
  for (int idx = tid; idx < K * D; idx += NTU_CTA) {
    int i = idx / D, q = idx % D;
    const double sv = sm.S.s[q], rs = mode == 2 ? sqrt(sv) : 1.0;
    const double2 ph = sm.ph[q];
    sm.MA[idx] = cscale(cmul(sm.S.W[q * 32 + i], ph), mode == 2 ? rs : sv);
    sm.MB[idx] = cscale(cmul(sm.S.A[q * 32 + i], cconj(ph)), rs);
  }
  __syncthreads();
  return 1;
}

// Tilt of a half sweep by a QR factorisation (Fig. 5(a)).  Before the step
// that solves for one factor, the other, fixed one is brought to an
// isometry: Y = Q R with Q (K x D) orthonormal and R upper triangular with
// a real positive diagonal (classical Gram-Schmidt, a column orthogonalised
// a second time only when the first pass removed more than half of its
// squared norm), Y <- Q and the free factor Z <- Z R^T, so the bond
// matrix Z Y^T is unchanged.  Any isometry spanning the columns of Y serves:
// the reduced metric for Q W (W unitary) is (1 x W)^H g_A (1 x W), with the
// same spectrum, pseudo-inverse truncation and minimiser Z Y^T; only the
// last tilt (the balance) fixes the gauge, by the SVD.  side 0 (A step):
// Y = M_B, Z = M_A; side 1: Y = M_A, Z = M_B.  Returns 0, changing nothing,
// when min R_qq <= 1e-12 max R_qq (the SVD tilt then handles the nearly
// rank-deficient factor).  Gram-Schmidt takes D dependent reductions where
// the one-sided Jacobi SVD takes some 15 rounds of FP64 rotations.
static __device__ int als_tilt_qr(AlsShared& sm, const AlsArgs& a, int side) {
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31, K = a.K, D = a.D;
  double2* Y = side == 0 ? sm.MB : sm.MA;
  double2* Z = side == 0 ? sm.MA : sm.MB;
  double2* Q = sm.S.A;                                  // column q at Q[q * 32 + i]
  double2* R = sm.S.V;                                  // R[p * 32 + q], row p, column q
  double* rd = sm.S.s;                                  // R_qq
  for (int idx = tid; idx < 32 * D; idx += NTU_CTA) {
    const int i = idx & 31, q = idx >> 5;
    Q[idx] = i < K ? Y[i * D + q] : cz();
    R[q * 32 + i] = cz();                               // rows q < D, columns i < 32
  }
  __syncthreads();
  // squared column norms before any projection (warp per column)
  double* n2 = sm.S.s + 8;
  for (int q = wid; q < D; q += NTU_WARPS) {
    double s2 = lid < K ? cabs2(Q[q * 32 + lid]) : 0.0;
    s2 = warp_sum(s2);
    if (lid == 0) n2[q] = s2;
  }
  __syncthreads();
  for (int q = 0; q < D; ++q) {
    // project out the previous columns; a second pass only when the first
    // left less than 1/sqrt(2) of the norm (the DGKS criterion: then the
    // column is orthogonal to working precision)
    double before = n2[q];
    for (int pass = 0; pass < 2 && q > 0; ++pass) {
      // c_p = Q_p^H v for p < q (warp p), then v -= sum_p Q_p c_p
      for (int p = wid; p < q; p += NTU_WARPS) {
        double2 c = lid < K ? cmulc(Q[p * 32 + lid], Q[q * 32 + lid]) : cz();
        c = warp_sum2(c);
        if (lid == 0) {
          sm.ph[p] = c;
          R[p * 32 + q] = cadd(R[p * 32 + q], c);
        }
      }
      __syncthreads();
      if (tid < K) {
        double2 v = Q[q * 32 + tid];
        for (int p = 0; p < q; ++p) v = cfms(Q[p * 32 + tid], sm.ph[p], v);
        Q[q * 32 + tid] = v;
      }
      __syncthreads();
      if (wid == 0) {
        double s2 = lid < K ? cabs2(Q[q * 32 + lid]) : 0.0;
        s2 = warp_sum(s2);
        if (lid == 0) n2[q] = s2;
      }
      __syncthreads();
      const double after = n2[q];
      if (after >= 0.5 * before) break;
      before = after;
    }
    const double rq = sqrt(n2[q]);
    if (tid < K) Q[q * 32 + tid] = rq > 0.0 ? cscale(Q[q * 32 + tid], 1.0 / rq) : cz();
    if (tid == 0) {
      R[q * 32 + q] = make_double2(rq, 0.0);
      rd[q] = rq;
    }
    __syncthreads();
  }
  double lo = rd[0], hi = rd[0];
  for (int q = 1; q < D; ++q) {
    lo = rd[q] < lo ? rd[q] : lo;
    hi = rd[q] > hi ? rd[q] : hi;
  }
  if (!(lo > 1e-12 * hi) || !isfinite(hi)) return 0;
  // Z R^T into W, then both factors in place
  for (int idx = tid; idx < K * D; idx += NTU_CTA) {
    const int i = idx / D, q = idx % D;
    double2 acc = cz();
    for (int p = q; p < D; ++p) acc = cfma(Z[i * D + p], R[q * 32 + p], acc);
    sm.S.W[idx] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < K * D; idx += NTU_CTA) {
    Z[idx] = sm.S.W[idx];
    Y[idx] = Q[(idx % D) * 32 + idx / D];
  }
  __syncthreads();
  return 1;
}

// als_reduced in double-FP32 arithmetic, block by block: block (f1, f),
// f1 >= f, of the reduced metric is
//   gX[(f1,q1),(f,q)] = sum_{c',c} conj(F[c'][q1]) g[f1*sf + c'*sc][f*sf + c*sc] F[c][q],
// a K x K block of g contracted with F on both sides.  One warp takes a
// block: T = g_blk F (K x D) goes to a warp-private tile in the SVD arrays A
// and V (free between tilts), then F^H T gives the D x D block, written to
// gX in FP64 (scaled back by 2^e) and to gXdf in double-FP32 (for the matrix
// products of the conjugate-gradient solve), mirrored into the upper
// triangle.  Every element of g is read once per call and no intermediate
// leaves the SM.  F (the isometric factor) is split into als_fdf(sm).
// When an item's ALS runs on `split` CTAs, CTA `rank` builds every
// split-th block and writes it into all `split` private copies of gX and
// gXdf (`cstride` elements apart, the first at gX, gXdf).
template <bool SPLIT>
static __device__ void als_reduced_df(AlsShared& sm, const AlsArgs& a, const float4* gdf,
                                      const float4* gdfT, int e, int side, double2* gX, float4* gXdf,
                                      int rank_, int split_, long long cstride) {
  const int rank = SPLIT ? rank_ : 0, split = SPLIT ? split_ : 1;
  const int tid = threadIdx.x, K = a.K, D = a.D, ng = a.ng, nA = a.nA;
  const int warp = tid >> 5, lane = tid & 31;
  const double2* F = side == 0 ? sm.MB : sm.MA;
  // the B step reads the block (f1, f) of g with rows (c', f1) and columns
  // (c, f) as rows f1*K + c' and columns f*K + c of gdfT
  const float4* gb = side == 0 ? gdf : gdfT;
  const int nq = (D + 3) >> 2;
  const float4* Fd = als_fdf(sm);
  float4* Tw = reinterpret_cast<float4*>(sm.S.A) + warp * (32 * 8);   // K x D <= 256
  for (int i = tid; i < K * D; i += NTU_CTA) als_fdf(sm)[i] = df_split(F[i]);
  __syncthreads();
  const int nblk = K * (K + 1) / 2;
  for (int blk = warp + NTU_WARPS * rank; blk < nblk; blk += NTU_WARPS * split) {
    int f1 = (int)((sqrtf(8.0f * (float)blk + 1.0f) - 1.0f) * 0.5f);
    while ((f1 + 1) * (f1 + 2) / 2 <= blk) ++f1;
    while (f1 > 0 && f1 * (f1 + 1) / 2 > blk) --f1;
    const int f = blk - f1 * (f1 + 1) / 2;
    // T[c'][q] = sum_c g[f1*sf + c'*sc][f*sf + c*sc] F[c][q] (sf = K, sc = 1
    // on the A step, sf = 1, sc = K on the B step), four q per item
    for (int it = lane; it < K * nq; it += 32) {
      const int c1 = it / nq, q0 = (it % nq) * 4;
      const float4* gr = gb + (size_t)(f1 * K + c1) * ng + f * K;
      float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0, acc2 = acc0, acc3 = acc0;
#pragma unroll 4
      for (int c = 0; c < K; ++c) {
        const float4 gv = gr[c];
        const float4* Fc = Fd + c * D + q0;
        df_cmac<false>(acc0, gv, Fc[0]);
        if (q0 + 1 < D) df_cmac<false>(acc1, gv, Fc[1]);
        if (q0 + 2 < D) df_cmac<false>(acc2, gv, Fc[2]);
        if (q0 + 3 < D) df_cmac<false>(acc3, gv, Fc[3]);
      }
      float4* out = Tw + c1 * D + q0;
      out[0] = acc0;
      if (q0 + 1 < D) out[1] = acc1;
      if (q0 + 2 < D) out[2] = acc2;
      if (q0 + 3 < D) out[3] = acc3;
    }
    __syncwarp();
    // block[q1][q] = sum_c' conj(F[c'][q1]) T[c'][q]; the diagonal block keeps
    // q1 >= q and mirrors it, so gX is Hermitian to the last bit
    for (int it = lane; it < D * D; it += 32) {
      const int q1 = it / D, q = it % D;
      if (f1 == f && q1 < q) continue;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
      for (int c1 = 0; c1 < K; ++c1) df_cmac<true>(acc, Fd[c1 * D + q1], Tw[c1 * D + q]);
      const int row = f1 * D + q1, col = f * D + q;
      double2 v = df_join(acc);
      if (e != 0) v = make_double2(scalbn(v.x, e), scalbn(v.y, e));
      for (int cp = 0; cp < split; ++cp) {
        double2* gXc = gX + cp * cstride;
        float4* gXdfc = gXdf + cp * cstride;
        gXc[(size_t)col * nA + row] = v;
        gXdfc[(size_t)col * nA + row] = acc;
        if (row != col) {                                // upper triangle
          gXc[(size_t)row * nA + col] = cconj(v);
          gXdfc[(size_t)row * nA + col] = make_float4(acc.x, -acc.y, acc.z, -acc.w);
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// als_reduced_df with its first stage, T = g_blk F, on the tensor cores
// (oz_build.cuh).  Thread 0 issues the TMA loads of the g slices (three
// 16 KB boxes per tile, two buffers) and the MMAs; all eight warps combine
// the six accumulator levels into the double-FP32 tile of T in shared
// memory (warp w: TMEM lanes of quarter w % 4, output columns of half w / 4)
// and then form the D x D blocks F^H T of the tile's row blocks f1 >= f, one
// block per warp.  Per tile, as soon as its accumulator is complete both
// buffers are free and the next tile's first two boxes are loaded; their
// MMAs go out after the epilogue, the third box is loaded while the blocks
// are formed and issued after them, so the loads overlap the lane work.
// Returns false if a tensor-core wait ran out (status raised, loads in
// flight drained; the caller then uses the lane build).
template <int KK>
static __device__ bool als_reduced_oz(AlsShared& sm, const AlsArgs& a, const CUtensorMap* mapG,
                                      long long item, int e, int side, double2* gX, float4* gXdf,
                                      const short* gexp, uint32_t tmem, int rank, int split,
                                      long long cstride) {
  constexpr int K = KK, ng = K * K;                   // K = D r, fixed per instantiation
  const int tid = threadIdx.x, D = a.D, nA = a.nA;
  const int warp = tid >> 5, lane = tid & 31;
  const OzGeo Gm = oz_geo(K);
  const double2* F = side == 0 ? sm.MB : sm.MA;
  const OzSmem os = oz_smem(&sm.S, sm.red);
  float4* Ts = reinterpret_cast<float4*>(sm.y);        // 128 rows x D (y, y2, p, ap: 16 KB)
  uint64_t* full = os.bar;
  uint64_t* freeb = os.bar + 2;
  uint64_t* accb = os.bar + 4;
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) tc::mbar_init(&os.bar[i], 1);
    tc::fence_barrier_init();
    *os.dead = 0;
  }
  oz_fill_b(os, F, K, D);                               // ends with a barrier
  // ---- thread 0's steps.  Box G (tile G / 3, box G % 3) uses buffer G & 1,
  // whose use number G >> 1 gives the barrier phases.  `issued` / `landed`
  // count the boxes loaded and waited for, so that a failed wait can still
  // drain the loads in flight before the shared memory is reused.
  int issued = 0, landed = 0;
  bool ok0 = true;
  const uint64_t bd = tc::sdesc_k128(tc::smem_u32(os.bop));
  // this CTA's tiles: tau = rank + j split, j = 0 .. nt - 1 (all of them
  // unless an item's ALS runs on a cluster); G counts this CTA's boxes
  const int nt = (Gm.ntiles - rank + split - 1) / split;
  auto load = [&](int G) {
    int f, t;
    oz_tile_ft(Gm, rank + (G / Gm.boxes) * split, f, t);
    ++issued;
    tc::mbar_expect_tx(&full[G & 1], OZ_BOX_BYTES);
    tc::tma_load_3d(os.abuf + (G & 1) * OZ_BOX_BYTES, mapG, &full[G & 1], 0,
                    (int)oz_row(Gm, side, f, t, G % Gm.boxes), (int)item);
  };
  auto mma_box = [&](int G) {
    if (!ok0) return;
    if (!tc::mbar_wait_sleep(&full[G & 1], (uint32_t)((G >> 1) & 1), OZ_POLLS)) { ok0 = false; return; }
    ++landed;
    tc::fence_after_sync();
    const uint64_t ad = tc::sdesc_k128(tc::smem_u32(os.abuf + (G & 1) * OZ_BOX_BYTES));
    const int box = G % Gm.boxes;
    // slice i = box spb + h sits at byte 4 K h of the box row; a K = 16
    // step advances the descriptors by 32 bytes (2 in units of 16)
    for (int h = 0; h < Gm.spb; ++h) {
      const int i = box * Gm.spb + h;
      const uint32_t idesc = tc::idesc_bf16_f32(128, (OZ_SLICES - i) * OZ_LEVEL_COLS);
      for (int kk = 0; kk < Gm.ksteps; ++kk)
        tc::mma_bf16(tmem + (uint32_t)(i * OZ_LEVEL_COLS), ad + (K / 4) * h + 2 * kk,
                     bd + 2 * kk, idesc, (i | kk) != 0);
    }
    tc::mma_commit(&freeb[G & 1]);
    if (box == Gm.boxes - 1) tc::mma_commit(accb);
  };
  auto wait_free = [&](int G) {       // the MMAs of box G have retired
    if (ok0 && !tc::mbar_wait_sleep(&freeb[G & 1], (uint32_t)((G >> 1) & 1), OZ_POLLS)) ok0 = false;
  };
  if (tid == 0 && nt > 0) {                           // tile 0 in full
    load(0);
    load(1);
    for (int b = 0; b < Gm.boxes; ++b) {
      mma_box(b);
      if (b + 2 < Gm.boxes) {
        wait_free(b);
        if (ok0) load(b + 2);
      }
    }
    if (!ok0) *os.dead = 1;
  }
  __syncthreads();
  for (int j = 0; j < nt && !*os.dead; ++j) {
    int f, t;
    oz_tile_ft(Gm, rank + j * split, f, t);
    const int tau = j;                                 // accumulator phase
    const int Gn = (j + 1) * Gm.boxes;                 // first box of the next tile
    const bool more = j + 1 < nt;
    // ---- epilogue: warp w combines the six levels of TMEM lane row =
    // 32 (w % 4) + lane for the output columns of q = 4 (w / 4) .. + 3
    {
      const bool ready =
          __all_sync(0xffffffffu, tc::mbar_wait_sleep(accb, (uint32_t)(tau & 1), OZ_POLLS));
      tc::fence_after_sync();
      if (tid == 0 && ready && more && ok0) {
        // every MMA of this tile has retired: both buffers take the next
        // tile's first two boxes now
        load(Gn);
        load(Gn + 1);
      }
      const int row = (warp & 3) * 32 + lane, qh = warp >> 2;
      float hi[8], lo[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) { hi[m] = 0.f; lo[m] = 0.f; }
      if (ready) {
        const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(qh * 8);
#pragma unroll
        for (int l0 = 0; l0 < OZ_SLICES; l0 += 3) {
          float v[24];
          tc::tmem_ld8x3(ta + l0 * OZ_LEVEL_COLS, ta + (l0 + 1) * OZ_LEVEL_COLS,
                         ta + (l0 + 2) * OZ_LEVEL_COLS, v);
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const float sc = __int_as_float((127 - 8 * (l0 + u + 2)) << 23);   // 2^-8(l+2)
#pragma unroll
            for (int m = 0; m < 8; ++m) df_add1(hi[m], lo[m], v[u * 8 + m] * sc, 0.f);
          }
        }
      } else {
        *os.dead = 1;
      }
      // exponents are relative to the unscaled g: T in the frame g 2^-ge
      const int er = gexp[(side * K + f) * ng + t * 128 + row] - e;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = qh * 4 + j;
        if (q < D) {
          const int ex = er + os.eq[q];
          if (ex > -126 && ex < 128) {                  // 2^ex as a normal FP32: exact products
            const float sc = __int_as_float((ex + 127) << 23);
            Ts[row * D + q] = make_float4(hi[2 * j] * sc, hi[2 * j + 1] * sc, lo[2 * j] * sc,
                                          lo[2 * j + 1] * sc);
          } else {
            Ts[row * D + q] = make_float4(ldexpf(hi[2 * j], ex), ldexpf(hi[2 * j + 1], ex),
                                          ldexpf(lo[2 * j], ex), ldexpf(lo[2 * j + 1], ex));
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (*os.dead) break;
    // ---- the next tile's boxes go out but its last, which loads meanwhile
    if (tid == 0 && more) {
      tc::fence_after_sync();
      for (int b = 0; b + 1 < Gm.boxes; ++b) {
        mma_box(Gn + b);
        if (b + 2 <= Gm.boxes - 1) {
          wait_free(Gn + b);
          if (ok0) load(Gn + b + 2);
        }
      }
    }
    // ---- second stage: the entries (q1, q) of the blocks (f1, f) of this
    // tile with f1 >= f, spread over the threads (block f1 from rows
    // 16 (f1 - 8 t) .. of the tile)
    const int fa = f > t * Gm.bpt ? f : t * Gm.bpt;    // first row block with f1 >= f
    const int nent = ((t + 1) * Gm.bpt - fa) * D * D;
    const float4* Fd = os.fdf;
    // warp 0 issues the loads and MMAs meanwhile: warps 1-7 take the entries
    for (int it = tid - 32; it < nent; it += NTU_CTA - 32) {
      if (it < 0) break;
      const int f1 = fa + it / (D * D), q1 = (it % (D * D)) / D, q = it % D;
      if (f1 == f && q1 < q) continue;
      {
        const float4* Tw = Ts + (f1 - t * Gm.bpt) * K * D;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
        for (int c1 = 0; c1 < K; ++c1) df_cmac<true>(acc, Fd[c1 * D + q1], Tw[c1 * D + q]);
        const int row = f1 * D + q1, col = f * D + q;
        double2 v = df_join(acc);
        if (e != 0) v = make_double2(scalbn(v.x, e), scalbn(v.y, e));
        for (int cp = 0; cp < split; ++cp) {             // every CTA's copy
          double2* gXc = gX + cp * cstride;
          float4* gXdfc = gXdf + cp * cstride;
          gXc[(size_t)col * nA + row] = v;
          gXdfc[(size_t)col * nA + row] = acc;
          if (row != col) {
            gXc[(size_t)row * nA + col] = cconj(v);
            gXdfc[(size_t)row * nA + col] = make_float4(acc.x, -acc.y, acc.z, -acc.w);
          }
        }
      }
    }
    if (tid == 0 && more) {
      mma_box(Gn + Gm.boxes - 1);                      // completes the next accumulator
      if (!ok0) *os.dead = 1;
    }
    __syncthreads();
  }
  const bool ok = !*os.dead;
  __syncthreads();
  if (tid == 0 && !ok) {
    for (int G = landed; G < issued; ++G)               // drain the loads in flight
      tc::mbar_wait(&full[G & 1], (uint32_t)((G >> 1) & 1), OZ_WAIT);
    raise_status(a.status, ST_TIMEOUT, WHY_TC_WAIT);
  }
  __syncthreads();
  return ok;
}

// Reduced metric and source for the free side (Fig. 5(b,c)).  side 0: the
// A step, free index i of (i, j), fixed F = MB; side 1: the B step, free j,
// F = MA.  gX is written column-major (nA x nA), J into a.jv.
static __device__ void als_reduced(AlsShared& sm, const AlsArgs& a, const double2* g, int side,
                                   double2* Tm, double2* gX, double2* jv, const double2* gx0) {
  const int tid = threadIdx.x, K = a.K, D = a.D, ng = a.ng, nA = a.nA;
  const double2* F = side == 0 ? sm.MB : sm.MA;
  const int sf = side == 0 ? K : 1, sc = side == 0 ? 1 : K;
  // Tm[r][(f,q)] = sum_c g[r][f*sf + c*sc] F[c][q], only where the free
  // index of row r is >= f: the lower triangle of gX below reads no other
  for (int idx = tid; idx < ng * nA; idx += NTU_CTA) {
    int r = idx / nA, fq = idx % nA, f = fq / D, q = fq % D;
    if ((side == 0 ? r / K : r % K) < f) continue;
    const double2* gr = g + (size_t)r * ng + f * sf;
    double2 acc = cz();
    for (int c = 0; c < K; ++c) acc = cfma(gr[c * sc], F[c * D + q], acc);
    Tm[idx] = acc;
  }
  __syncthreads();
  // gX[(f',q'),(f,q)] = sum_c' conj(F[c'][q']) Tm[f'*sf + c'*sc][(f,q)] from
  // the lower triangle, mirrored into the upper one
  for (int idx = tid; idx < nA * nA; idx += NTU_CTA) {
    int col = idx / nA, row = idx % nA, f1 = row / D, q1 = row % D;
    if (row < col) continue;
    double2 acc = cz();
    for (int c = 0; c < K; ++c)
      acc = cfmac(F[c * D + q1], Tm[(size_t)(f1 * sf + c * sc) * nA + col], acc);
    gX[idx] = acc;
    if (row != col) gX[(size_t)row * nA + col] = cconj(acc);
  }
  __syncthreads();
}

// Source J of the free side: J[(f,q)] = sum_c conj(F[c][q]) (g x0)[f*sf + c*sc].
static __device__ void als_source(AlsShared& sm, const AlsArgs& a, int side, double2* jv,
                                  const double2* gx0) {
  const int K = a.K, D = a.D, nA = a.nA;
  const double2* F = side == 0 ? sm.MB : sm.MA;
  const int sf = side == 0 ? K : 1, sc = side == 0 ? 1 : K;
  for (int row = threadIdx.x; row < nA; row += NTU_CTA) {
    int f1 = row / D, q1 = row % D;
    double2 acc = cz();
    for (int c = 0; c < K; ++c) acc = cfmac(F[c * D + q1], gx0[f1 * sf + c * sc], acc);
    jv[row] = acc;
  }
  __syncthreads();
}

// Certified shortcut of the tolerance selection.  With B >= lambda_max of gX
// and tau_max the largest candidate, a proof that lambda_min > sigma =
// (tau_max + 1e-12) B (the 1e-12 B margin covers rounding) means every
// candidate tolerance keeps every eigenpair: all candidates give the same
// eps, the selection rule returns tau_max, and the pseudo-inverse is the
// inverse.  Two proofs are tried in turn.  Tier 1: the Gershgorin discs
// (B = max_i d_i + s_i) lie right of sigma; M = gX^{-1} J then comes from
// conjugate gradients.  Tier 2: gX - sigma I has a Cholesky factor L L^H;
// M then follows from the fixed-point iteration (L L^H) v_{k+1} = J -
// sigma v_k (its fixed point solves gX v = J), which contracts by
// sigma / (lambda_min - sigma).  Both read the lower triangle of gX (tier 1
// mirrors it into the upper one).  Returns 1 when solved, 0 when neither
// proof holds or an iteration stalls; the caller then takes the eigen path.
static __device__ void als_mirror(double2* gX, int nA);

// Upper triangle of the double-FP32 copy from its lower triangle.
static __device__ void als_mirror_df(float4* A, int nA) {
  for (int idx = threadIdx.x; idx < nA * nA; idx += NTU_CTA) {
    const int col = idx / nA, row = idx % nA;
    if (row < col) {
      const float4 v = A[(size_t)row * nA + col];
      A[idx] = make_float4(v.x, -v.y, v.z, -v.w);
    }
  }
  __syncthreads();
}

// out = g_A v (g_A full, column-major), in FP64 or, with df, in double-FP32
// on the copy scaled by 2^-ge (v is split into als_pdf(sm) first).  Two threads
// per row take the two halves of the sum, each with two independent
// accumulators, so that the dependent chains are a quarter of n_A long.
// With rsum (df only), also rsum[i] = sum_{j != i} |Re| + |Im| of the high
// parts of row i, summed in FP32 (the Gershgorin radii of the solve).
static __device__ void als_matvec(AlsShared& sm, const double2* A, const float4* Adf, const double2* v,
                                  double2* out, int nA, bool df, float* rsum = nullptr) {
  const int tid = threadIdx.x, h = tid & 1;
  const int half = (nA + 1) >> 1;
  const int j0 = h ? half : 0, j1 = h ? nA : half;
  if (df) {
    for (int i = tid; i < nA; i += NTU_CTA) als_pdf(sm)[i] = df_split(v[i]);
    __syncthreads();
  }
  for (int base = 0; base < nA; base += NTU_CTA / 2) {
    const int i = base + (tid >> 1);
    const bool on = i < nA;
    if (df) {
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
      float sr = 0.f;
      if (on) {
        int j = j0;
        if (rsum) {
#pragma unroll 4
          for (; j + 1 < j1; j += 2) {
            const float4 e0 = Adf[(size_t)j * nA + i], e1 = Adf[(size_t)(j + 1) * nA + i];
            df_cmac<false>(a0, e0, als_pdf(sm)[j]);
            df_cmac<false>(a1, e1, als_pdf(sm)[j + 1]);
            sr += (j != i ? fabsf(e0.x) + fabsf(e0.y) : 0.f) +
                  (j + 1 != i ? fabsf(e1.x) + fabsf(e1.y) : 0.f);
          }
          if (j < j1) {
            const float4 e0 = Adf[(size_t)j * nA + i];
            df_cmac<false>(a0, e0, als_pdf(sm)[j]);
            sr += j != i ? fabsf(e0.x) + fabsf(e0.y) : 0.f;
          }
        } else {
#pragma unroll 4
          for (; j + 1 < j1; j += 2) {
            df_cmac<false>(a0, Adf[(size_t)j * nA + i], als_pdf(sm)[j]);
            df_cmac<false>(a1, Adf[(size_t)(j + 1) * nA + i], als_pdf(sm)[j + 1]);
          }
          if (j < j1) df_cmac<false>(a0, Adf[(size_t)j * nA + i], als_pdf(sm)[j]);
        }
      }
      if (rsum) {
        sr += __shfl_xor_sync(0xffffffffu, sr, 1);
        if (on && h == 0) rsum[i] = sr;
      }
      df_add1(a0.x, a0.z, a1.x, a1.z);
      df_add1(a0.y, a0.w, a1.y, a1.w);
      const float4 o = make_float4(__shfl_xor_sync(0xffffffffu, a0.x, 1), __shfl_xor_sync(0xffffffffu, a0.y, 1),
                                   __shfl_xor_sync(0xffffffffu, a0.z, 1), __shfl_xor_sync(0xffffffffu, a0.w, 1));
      df_add1(a0.x, a0.z, o.x, o.z);
      df_add1(a0.y, a0.w, o.y, o.w);
      if (on && h == 0) {
        double2 r = df_join(a0);
        if (sm.ge != 0) r = make_double2(scalbn(r.x, sm.ge), scalbn(r.y, sm.ge));
        out[i] = r;
      }
    } else {
      double2 a0 = cz(), a1 = cz();
      if (on) {
        int j = j0;
#pragma unroll 4
        for (; j + 1 < j1; j += 2) {
          a0 = cfma(A[(size_t)j * nA + i], v[j], a0);
          a1 = cfma(A[(size_t)(j + 1) * nA + i], v[j + 1], a1);
        }
        if (j < j1) a0 = cfma(A[(size_t)j * nA + i], v[j], a0);
      }
      a0 = cadd(a0, a1);
      a0.x += __shfl_xor_sync(0xffffffffu, a0.x, 1);
      a0.y += __shfl_xor_sync(0xffffffffu, a0.y, 1);
      if (on && h == 0) out[i] = a0;
    }
  }
  __syncthreads();
}

static __device__ int als_solve_chol(AlsShared& sm, const AlsArgs& a, int side, double2* gX,
                                     double2* gC, const double2* jv, double tau_max) {
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31, nA = a.nA;
  // Gershgorin discs: d_i = Re gX[i][i] and s_i = sum_{j != i} (|Re| +
  // |Im|) >= sum_{j != i} |gX[i][j]|, so every eigenvalue lies in
  // [min(d - s), max(d + s)].  gX is full and Hermitian, so row i's sum is
  // column i's (contiguous).  On the mixed contexts s_i is summed in FP32
  // from the high parts of the double-FP32 copy (scaled by 2^-ge), in the
  // pass of the first product g_A x of the conjugate gradients below, which
  // reads every entry anyway (the product is dropped if tier 2 runs); that
  // rounding (< 1e-5 relative for n_A <= 256) is covered by inflating s_i by
  // 1e-4.
  const bool df = a.df != 0;
  const float4* gXdf = reinterpret_cast<const float4*>(gC);
  const double2* M0 = side == 0 ? sm.MA : sm.MB;
  double glo = INFINITY, ghi = -INFINITY;
  if (df) {
    float* rsum = reinterpret_cast<float*>(sm.S.V);         // free during a solve
    for (int i = tid; i < nA; i += NTU_CTA) sm.y[i] = M0[i];
    __syncthreads();
    als_matvec(sm, gX, gXdf, sm.y, sm.ap, nA, true, rsum);  // ap = g_A x, and the s_i
    for (int i = tid; i < nA; i += NTU_CTA) {
      const double sgi = scalbn((double)rsum[i], sm.ge) * (1.0 + 1e-4);
      const double d = gX[(size_t)i * nA + i].x;
      glo = fmin(glo, d - sgi);
      ghi = fmax(ghi, d + sgi);
    }
  } else {
    for (int i = wid; i < nA; i += NTU_WARPS) {
      const double2* col = gX + (size_t)i * nA;
      double sd = 0.0;
#pragma unroll 4
      for (int j = lid; j < nA; j += 32) {
        const double2 v = col[j];
        sd += j != i ? fabs(v.x) + fabs(v.y) : 0.0;
      }
      const double sgi = warp_sum(sd);
      const double d = gX[(size_t)i * nA + i].x;
      glo = fmin(glo, d - sgi);
      ghi = fmax(ghi, d + sgi);
    }
  }
  glo = block_min(glo, sm.red);
  const double bmax = block_max(ghi, sm.red);               // >= lambda_max
  if (!(bmax > 0.0) || !isfinite(bmax) || !isfinite(glo)) return 0;
  const double sigma = (tau_max + 1e-12) * bmax;
  if (glo > sigma) {
    // Tier 1: the discs alone prove lambda_min > tau_max lambda_max; solve
    // gX v = J by conjugate gradients on the full matrix, started from the
    // current factor (the tilt left it in the gauge of the fixed side, so
    // near convergence of the sweeps it already solves the system).  On the
    // mixed contexts the products g_A p run in double-FP32 on the copy the
    // build left in gC, and a candidate is accepted only once its residual,
    // recomputed in FP64, is <= 1e-13 |J| (at most three restarts from that
    // residual); the FP64 context iterates in FP64 down to 1e-15 |J|.
    if (!df) {
      for (int i = tid; i < nA; i += NTU_CTA) sm.y[i] = M0[i];
      __syncthreads();
      als_matvec(sm, gX, gXdf, sm.y, sm.ap, nA, false);     // ap = g_A x
    }
    double js = 0.0, rs = 0.0;
    for (int i = tid; i < nA; i += NTU_CTA) {
      const double2 r = csub(jv[i], sm.ap[i]);
      sm.y2[i] = r; sm.p[i] = r;
      js += cabs2(jv[i]);
      rs += cabs2(r);
    }
    js = block_sum(js, sm.red);
    rs = block_sum(rs, sm.red);
    const double stop = (df ? 1e-28 : 1e-30) * js;          // |r| <= 1e-14 (1e-15) |J|
    const double floor2 = (df ? 1e-24 : 1e-26) * js;        // rounding floor of the recursion
    const double accept = 1e-26 * js;                       // FP64 residual <= 1e-13 |J|
    int conv = 0, checks = 0;
    bool small = rs <= stop;
    double prev = rs;
    for (int it = 0; it < 80 && !conv; ++it) {
      if (small) {
        if (!df) { conv = 1; break; }
        als_matvec(sm, gX, gXdf, sm.y, sm.ap, nA, false);     // FP64 residual
        double r64 = 0.0;
        for (int i = tid; i < nA; i += NTU_CTA) {
          const double2 r = csub(jv[i], sm.ap[i]);
          sm.y2[i] = r; sm.p[i] = r;
          r64 += cabs2(r);
        }
        r64 = block_sum(r64, sm.red);
        if (r64 <= accept) { conv = 1; break; }
        if (++checks > 3) break;
        rs = r64; prev = r64; small = false;
        continue;
      }
      als_matvec(sm, gX, gXdf, sm.p, sm.ap, nA, df);
      double pap = 0.0;
      for (int i = tid; i < nA; i += NTU_CTA) pap += cmulc(sm.p[i], sm.ap[i]).x;
      pap = block_sum(pap, sm.red);
      if (!(pap > 0.0)) break;
      const double alpha = rs / pap;
      double rn = 0.0;
      for (int i = tid; i < nA; i += NTU_CTA) {
        double2 x = sm.y[i], r = sm.y2[i], p = sm.p[i], q = sm.ap[i];
        x.x = fma(alpha, p.x, x.x); x.y = fma(alpha, p.y, x.y);
        r.x = fma(-alpha, q.x, r.x); r.y = fma(-alpha, q.y, r.y);
        sm.y[i] = x; sm.y2[i] = r;
        rn += cabs2(r);
      }
      rn = block_sum(rn, sm.red);
      // converged, or stalled at the rounding floor of the recursion
      small = rn <= stop || (it >= 2 && rn > 0.25 * prev && rn <= floor2);
      prev = rn;
      const double beta = rn / rs;
      rs = rn;
      for (int i = tid; i < nA; i += NTU_CTA) {
        double2 r = sm.y2[i], p = sm.p[i];
        sm.p[i] = make_double2(fma(beta, p.x, r.x), fma(beta, p.y, r.y));
      }
      __syncthreads();
      if (small && !df) { conv = 1; break; }
    }
    if (conv) {
      double2* M = side == 0 ? sm.MA : sm.MB;
      for (int i = tid; i < nA; i += NTU_CTA) M[i] = sm.y[i];
      if (tid == 0) { sm.tau_sel = tau_max; sm.n_cg += 1; }
      __syncthreads();
      return 1;
    }
    __syncthreads();
  }
  // Tier 2: a Cholesky factorisation of gX - sigma I proves the same bound.
  for (int idx = tid; idx < nA * nA; idx += NTU_CTA)
    if (idx % nA >= idx / nA) gC[idx] = gX[idx];
  __syncthreads();
  if (!cta_cholesky(gC, nA, sigma, &sm.flag)) return 0;
  if (wid == 0) {
    const double2* M0 = side == 0 ? sm.MA : sm.MB;
    for (int i = lid; i < nA; i += 32) sm.y[i] = M0[i];     // warm start
    __syncwarp();
    int conv = 0;
    double prev = INFINITY;
    for (int it = 0; it < 60 && !conv; ++it) {
      for (int i = lid; i < nA; i += 32) {
        double2 v = sm.y[i], j = jv[i];
        sm.y2[i] = make_double2(fma(-sigma, v.x, j.x), fma(-sigma, v.y, j.y));
      }
      __syncwarp();
      warp_cholesky_solve(gC, nA, sm.y2);
      double diff = 0.0, vmax = 0.0;
      for (int i = lid; i < nA; i += 32) {
        double2 n = sm.y2[i], o = sm.y[i];
        diff = fmax(diff, fabs(n.x - o.x) + fabs(n.y - o.y));
        vmax = fmax(vmax, fabs(n.x) + fabs(n.y));
        sm.y[i] = n;
      }
      diff = warp_max(diff);
      vmax = warp_max(vmax);
      __syncwarp();
      if (diff <= 1e-15 * vmax) conv = 1;                         // converged
      else if (it >= 3 && diff >= 0.5 * prev && diff <= 1e-13 * vmax) conv = 1;  // rounding floor
      prev = diff;
    }
    if (lid == 0) sm.flag = conv;
  }
  __syncthreads();
  if (!sm.flag) return 0;
  double2* M = side == 0 ? sm.MA : sm.MB;
  for (int i = tid; i < nA; i += NTU_CTA) M[i] = sm.y[i];
  if (tid == 0) { sm.tau_sel = tau_max; sm.n_fast += 1; }
  __syncthreads();
  return 1;
}

// Fill the upper triangle of gX from its lower triangle (the eigen path
// works on full storage).
static __device__ void als_mirror(double2* gX, int nA) {
  for (int idx = threadIdx.x; idx < nA * nA; idx += NTU_CTA) {
    int col = idx / nA, row = idx % nA;
    if (row < col) gX[idx] = cconj(gX[(size_t)row * nA + col]);
  }
  __syncthreads();
}

// M = pinv_tau(gX) J with the tolerance of the grid that minimises
// eps(tau) = eps0 - sum_{lambda_i > tau lambda_max} |y_i|^2 / lambda_i,
// y = W^H J (Eq. 4 inserted in Eq. 3); ties within 1e-14 eps0 go to the
// larger tau.  The result is written to sm.MA (side 0) or sm.MB (side 1).
static __device__ void als_solve(AlsShared& sm, const AlsArgs& a, int side, double2* gX,
                                 const double2* jv, double2* pv, double2* tauv, double* dv, double* ev,
                                 RotLog& log) {
  const int tid = threadIdx.x, nA = a.nA;
  for (int i = tid; i < nA; i += NTU_CTA) sm.y[i] = jv[i];
  __syncthreads();
  cta_hetrd(gX, nA, dv, ev, tauv, pv, sm.red);
  cta_apply_q(gX, nA, tauv, sm.y, true, sm.red);
  if (tid == 0) {
    int st = tridiag_qr(dv, ev, nA, log, sm.y);
    if (st) sm.err |= WHY_ALS_QR;
    double lmax = dv[0];
    for (int i = 1; i < nA; ++i) lmax = fmax(lmax, dv[i]);
    int kmin = a.kmin < 0 ? 0 : a.kmin, kmax = a.kmax > 20 ? 20 : a.kmax;
    double tsel = als_tau(kmin);
    if (lmax > 0.0 && !st) {
      double emin = INFINITY;
      for (int k = kmin; k <= kmax; ++k) {
        double thr = als_tau(k) * lmax, s = 0.0;
        for (int i = 0; i < nA; ++i)
          if (dv[i] > thr) s += cabs2(sm.y[i]) / dv[i];
        emin = fmin(emin, sm.eps0 - s);
      }
      for (int k = kmin; k <= kmax; ++k) {
        double thr = als_tau(k) * lmax, s = 0.0;
        for (int i = 0; i < nA; ++i)
          if (dv[i] > thr) s += cabs2(sm.y[i]) / dv[i];
        if (sm.eps0 - s <= emin + 1e-14 * sm.eps0) { tsel = als_tau(k); break; }
      }
      double thr = tsel * lmax;
      for (int i = 0; i < nA; ++i)
        sm.y[i] = dv[i] > thr ? cscale(sm.y[i], 1.0 / dv[i]) : cz();
      rotlog_apply_z(log, sm.y);
    } else {
      for (int i = 0; i < nA; ++i) sm.y[i] = cz();
    }
    sm.tau_sel = tsel;
    sm.n_eig += 1;
  }
  __syncthreads();
  cta_apply_q(gX, nA, tauv, sm.y, false, sm.red);
  double2* M = side == 0 ? sm.MA : sm.MB;
  for (int i = tid; i < nA; i += NTU_CTA) M[i] = sm.y[i];
  __syncthreads();
}

// MINB: CTAs per SM the register budget is sized for (2: 128 registers, no
// spills; 3: 80 registers, for batches of more than two items per SM).
// OZK: 0 for the lane build only; 16 or 32 for the instantiations with the
// tensor-core build at that K (kept out of the other instantiations, whose
// register allocation it would perturb, and with K fixed at compile time).
template <int MINB, bool SPLIT, int OZK>
__global__ void __launch_bounds__(NTU_CTA, MINB) k_als(AlsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AlsShared& sm = *reinterpret_cast<AlsShared*>(smem_raw);
  const int tid = threadIdx.x, wid = tid >> 5, lid = tid & 31;
  // an item's ALS runs on a.split CTAs (one cluster, rank = position in it):
  // all of them carry out the whole ALS on identical data, each in its own
  // scratch copy (index vitem), so their control flow is identical; only
  // the reduced-metric build is divided between them, and rank 0 writes the
  // results
  const int split = SPLIT ? a.split : 1, rank = SPLIT ? (int)(blockIdx.x % split) : 0;
  const long long item = SPLIT ? blockIdx.x / split : blockIdx.x, vitem = blockIdx.x;
  const int K = a.K, D = a.D, ng = a.ng, nA = a.nA;
  const double2* g = a.g + item * (long long)ng * ng;
  const double2* RA = a.RA + item * K * K;
  const double2* RB = a.RB + item * K * K;
  double2* x0 = a.x0 + vitem * ng;
  double2* gx0 = a.gx0 + vitem * ng;
  double2* Tm = a.Tm + vitem * (long long)ng * nA;
  double2* gX = a.gA + vitem * (long long)nA * nA;
  double2* jv = a.jv + vitem * nA;
  double2* pv = a.pv + vitem * nA;
  double2* tauv = a.tauv + vitem * nA;
  double* dv = a.dv + vitem * nA;
  double* ev = a.ev + vitem * nA;
  RotLog log;
  log.c = a.rc + vitem * (long long)a.rotcap;
  log.s = a.rs + vitem * (long long)a.rotcap;
  log.k = a.rk + vitem * (long long)a.rotcap;
  log.cap = a.rotcap;
  log.count = 0;
  double2* gC = a.gC + vitem * (long long)nA * nA;
  const long long nA2 = (long long)nA * nA;
  double2* gX0 = a.gA + item * split * nA2;                 // the item's first copy
  double2* gC0 = a.gC + item * split * nA2;
  int phase = 0;
  const double tau_max = als_tau(a.kmin < 0 ? 0 : a.kmin);
  // tau_sel stays NaN when no solve runs (zero sweeps: the SVDU truncation)
  if (tid == 0) {
    sm.err = 0; sm.n_cg = 0; sm.n_fast = 0; sm.n_eig = 0; sm.ge = 0;
    sm.tau_sel = __longlong_as_double(0x7ff8000000000000ll);
  }
  // the tensor-core build (K = 16 or 32): its accumulator columns, held
  // until the last sweep (the address passes through red[0])
  const bool oz = OZK != 0 && a.oz && a.K == OZK;
  uint32_t oz_tmem = 0;
  if (oz) {
    if (wid == 0) tc::tmem_alloc(reinterpret_cast<uint32_t*>(sm.red), OZ_TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    oz_tmem = *reinterpret_cast<volatile uint32_t*>(sm.red);
    __syncthreads();
  }
  // X0 = R_A R_B^T, x0 = vec(X0) with kA slow
  for (int idx = tid; idx < K * K; idx += NTU_CTA) {
    int i = idx / K, j = idx % K;
    double2 acc = cz();
    for (int b = 0; b < K; ++b) acc = cfma(RA[i * K + b], RB[j * K + b], acc);
    x0[idx] = acc;
  }
  __syncthreads();
  const float4 *gdf = nullptr, *gdfT = nullptr;
  int ge = 0;
  if (a.df) {
    gdf = a.gdf + item * (long long)ng * ng;
    gdfT = a.gdfT + item * (long long)ng * ng;
    ge = a.gscale[item];                                   // g is split by k_gsplit
    if (tid == 0) sm.ge = ge;
  }
  // the slices of g come from k_oz_slice, launched before this kernel
  const short* gexp = oz ? a.gexp + item * (long long)2 * K * ng : nullptr;
  // gx0 = g x0 (double-FP32 products on the mixed contexts), eps0 = x0^H g x0
  double e0 = 0.0;
  if (a.df) {
    als_gmat_df(sm, a, gdf, ge, x0, gx0 - rank * (long long)ng, ng, ng, item, rank, split, phase);
    for (int r = tid; r < ng; r += NTU_CTA) e0 += cmulc(x0[r], gx0[r]).x;
  } else {
    for (int r = wid; r < ng; r += NTU_WARPS) {
      const double2* gr = g + (size_t)r * ng;
      double2 acc = cz();
      for (int c = lid; c < ng; c += 32) acc = cfma(gr[c], x0[c], acc);
      acc = warp_sum2(acc);
      if (lid == 0) {
        gx0[r] = acc;
        e0 += cmulc(x0[r], acc).x;
      }
    }
  }
  e0 = block_sum(e0, sm.red);
  if (tid == 0) sm.eps0 = e0;
  __syncthreads();
  // SVDU start (Fig. 2(c,d)).  X0 = U S V^H gives the balanced start
  // (U sqrt(S), conj(V) sqrt(S)) whose first tilt is (U S, conj(V)): with
  // sweeps to run, the start goes straight to the tilted pair.
  als_tilt(sm, a, a.sweeps > 0 ? 0 : 2, x0);
  bool tc_dead = false;
  for (int s = 0; s < a.sweeps && !tc_dead; ++s) {
    for (int side = 0; side < 2; ++side) {
      if ((s > 0 || side > 0) && !als_tilt_qr(sm, a, side) && !als_tilt_fast(sm, a, side))
        als_tilt(sm, a, side, nullptr);
      // every CTA of a cluster is done with its copy of the last reduced
      // metric before any writes the next one, and all blocks are in before
      // anyone reads
      if constexpr (OZK != 0) {
        if (split > 1) als_exchange(a, item, phase);
        const bool built = oz && als_reduced_oz<OZK>(sm, a, a.gmap, item, ge, side,
                                                     split > 1 ? gX0 : gX,
                                                     reinterpret_cast<float4*>(split > 1 ? gC0 : gC),
                                                     gexp, oz_tmem, rank, split, nA2);
        if (split > 1) als_exchange(a, item, phase);
        // a tensor-core wait that ran out has raised the status: this item's
        // ALS stops there (the accumulator is released at the end)
        if (!built) {
          if (!oz) raise_status(a.status, ST_NUMERIC, WHY_TC_WAIT);
          tc_dead = true;
          break;
        }
      } else if (a.df) {
        if (split > 1) als_exchange(a, item, phase);
        als_reduced_df<SPLIT>(sm, a, gdf, gdfT, ge, side, split > 1 ? gX0 : gX,
                              reinterpret_cast<float4*>(split > 1 ? gC0 : gC), rank, split, nA2);
        if (split > 1) als_exchange(a, item, phase);
      } else {
        als_reduced(sm, a, g, side, Tm, gX, jv, gx0);
      }
      als_source(sm, a, side, jv, gx0);
      if (!als_solve_chol(sm, a, side, gX, gC, jv, tau_max)) {
        als_mirror(gX, nA);
        als_solve(sm, a, side, gX, jv, pv, tauv, dv, ev, log);
      }
    }
  }
  if (OZK != 0 && a.oz && a.K == OZK) {
    // every MMA has retired before the accumulator columns are released
    const OzSmem os = oz_smem(&sm.S, sm.red);
    __syncthreads();
    if (tid == 0) {
      tc::mbar_init(&os.bar[5], 1);
      tc::fence_barrier_init();
      tc::mma_commit(&os.bar[5]);
      if (!tc::mbar_wait(&os.bar[5], 0, OZ_WAIT)) raise_status(a.status, ST_TIMEOUT, WHY_TC_WAIT);
    }
    __syncthreads();
    tc::fence_after_sync();
    if (wid == 0) tc::tmem_dealloc(oz_tmem & 0x7fffffffu, OZ_TMEM_COLS);
  }
  // balance (Fig. 5(d))
  if (a.sweeps > 0 && !als_tilt_fast(sm, a, 2)) als_tilt(sm, a, 2, nullptr);
  // eps = x^H g x, x = vec(MA MB^T) - x0
  double2* xv = Tm;
  for (int idx = tid; idx < ng; idx += NTU_CTA) {
    int i = idx / K, j = idx % K;
    double2 acc = cz();
    for (int q = 0; q < D; ++q) acc = cfma(sm.MA[i * D + q], sm.MB[j * D + q], acc);
    xv[idx] = csub(acc, x0[idx]);
  }
  __syncthreads();
  double eps = 0.0;
  if (a.df) {
    als_gmat_df(sm, a, gdf, ge, xv, gx0 - rank * (long long)ng, ng, ng, item, rank, split,
                phase);                                    // gx0 is free by now
    for (int r = tid; r < ng; r += NTU_CTA) eps += cmulc(xv[r], gx0[r]).x;
  } else {
    for (int r = wid; r < ng; r += NTU_WARPS) {
      const double2* gr = g + (size_t)r * ng;
      double2 acc = cz();
      for (int c = lid; c < ng; c += 32) acc = cfma(gr[c], xv[c], acc);
      acc = warp_sum2(acc);
      if (lid == 0) eps += cmulc(xv[r], acc).x;
    }
  }
  eps = block_sum(eps, sm.red);
  if (rank != 0) return;                                   // rank 0 writes the results
  double2* MAo = a.MA + item * K * D;
  double2* MBo = a.MB + item * K * D;
  for (int idx = tid; idx < K * D; idx += NTU_CTA) { MAo[idx] = sm.MA[idx]; MBo[idx] = sm.MB[idx]; }
  if (tid == 0) {
    double e0v = sm.eps0;
    double delta = e0v > 0.0 ? eps / e0v : 0.0;
    a.info[item * 4 + 0] = eps;
    a.info[item * 4 + 1] = delta;
    a.info[item * 4 + 2] = e0v;
    a.info[item * 4 + 3] = sm.tau_sel;
    if (sm.err || !isfinite(delta) || !isfinite(eps))
      raise_status(a.status, ST_NUMERIC, sm.err | ((!isfinite(delta) || !isfinite(eps)) ? WHY_ALS_NONFINITE : 0));
    if (a.path_counts) {
      atomicAdd(a.path_counts + 0, sm.n_cg);
      atomicAdd(a.path_counts + 1, sm.n_fast);
      atomicAdd(a.path_counts + 2, sm.n_eig);
    }
  }
}

// Sets the shared-memory limits of the instantiation and launches it: n
// items on `split` CTAs each (a cluster when split > 1), `three` selecting
// the 80-register budget of three CTAs per SM (single-CTA items only).
template <int OZK>
cudaError_t als_launch_impl(const AlsArgs& a, int n, int split, bool three, size_t smem,
                            cudaStream_t stream) {
  if (split > 1) {
    void (*ck)(AlsArgs) = k_als<2, true, OZK>;
    cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(ck, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(n * split), 1, 1);
    cfg.blockDim = dim3(NTU_CTA, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)split;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ck, a);
  }
  void (*kern)(AlsArgs) = three ? k_als<3, false, OZK> : k_als<2, false, OZK>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  kern<<<n, NTU_CTA, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace ntu
