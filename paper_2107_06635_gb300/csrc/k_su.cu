// Simple update (SU) of the two-site cell (Sec. II): the cell keeps a
// diagonal bond tensor lambda_b (D positive values) on each of its four
// inequivalent bonds, and the metric of a bond update is
// g_SU = 1_d (x) 1_d (x) prod_j lambda_j over the six outer bonds of the pair.
//
// The site tensors are held in the symmetric gauge: each leg carries
// sqrt(lambda) of its bond, so a pair contracted over its bond carries
// lambda_b once.  Weighting the three outer legs of each site by one more
// sqrt(lambda) puts the full lambda_j on the outer bonds; in the reduced
// space of the QR of those weighted tensors g_SU is the identity, and the
// minimiser of the error is the local SVD truncation (Fig. 2(c,d)) of
// R_A R_B^T.  The SU bond update is therefore: weight (k_su_weight), the
// gate + QR stage, the zero-sweep truncation with the identity metric
// (k_als), recompose, then remove the outer weights again (pseudo-inverse
// of lambda, k_su_weight) and set lambda_b to the kept singular values
// normalised to unit 2-norm (k_su_lambda).
#include "ntu_dev.cuh"
#include "ntu_impl.h"

namespace ntu {

// Bond carried by leg j in (l, u, r, dn) of the cell's site A and of B.
__constant__ int kSuBondsA[4] = {2, 1, 0, 3};
__constant__ int kSuBondsB[4] = {0, 3, 2, 1};

// Block 0: A -> Aout, block 1: B -> Bout.  Every leg whose bond is not
// `skip` is multiplied by sqrt(lambda) (inverse = 0) or by its
// pseudo-inverse (inverse = 1: values at or below 1e-14 x the bond's
// largest value give 0).  With `normalise`, the result is scaled to unit
// Frobenius norm.  In place is allowed (Aout == A).
__global__ void __launch_bounds__(NTU_CTA) k_su_weight(int dp, int D, int skip, int inverse,
                                                       int normalise, const double* __restrict__ lam,
                                                       const double2* A, const double2* B,
                                                       double2* Aout, double2* Bout) {
  __shared__ double w[4][8];
  __shared__ double sred[2 * NTU_WARPS];
  const int tid = threadIdx.x, site = blockIdx.x;
  const double2* T = site ? B : A;
  double2* out = site ? Bout : Aout;
  const int* bonds = site ? kSuBondsB : kSuBondsA;
  if (tid < 4) {
    const int b = bonds[tid];
    const double* lv = lam + b * D;
    double mx = 0.0;
    for (int i = 0; i < D; ++i) mx = fmax(mx, lv[i]);
    for (int i = 0; i < D; ++i) {
      double v = 1.0;
      if (b != skip) {
        if (!inverse) v = sqrt(lv[i]);
        else v = (lv[i] > 1e-14 * mx) ? 1.0 / sqrt(lv[i]) : 0.0;
      }
      w[tid][i] = v;
    }
  }
  __syncthreads();
  const int D2 = D * D, D3 = D2 * D, D4 = D3 * D;
  double nrm2 = 0.0;
  for (int idx = tid; idx < dp * D4; idx += NTU_CTA) {
    const int dn = idx % D, r = (idx / D) % D, u = (idx / D2) % D, l = (idx / D3) % D;
    const double f = w[0][l] * w[1][u] * w[2][r] * w[3][dn];
    const double2 v = cscale(T[idx], f);
    nrm2 += cabs2(v);
    out[idx] = v;
  }
  if (!normalise) return;
  const double nrm = sqrt(block_sum(nrm2, sred));
  const double sc = nrm > 0.0 ? 1.0 / nrm : 1.0;
  __syncthreads();
  for (int idx = tid; idx < dp * D4; idx += NTU_CTA) out[idx] = cscale(out[idx], sc);
}

// lambda_bond[q] = s_q / ||s||_2 with s_q = sum_i |M_A[i][q]|^2: after the
// balanced truncation M_A = U sqrt(S) (U with orthonormal columns), so the
// squared column norms are the kept singular values.  One warp.
__global__ void k_su_lambda(int K, int D, const double2* __restrict__ MA, double* lam, int bond) {
  const int lid = threadIdx.x;
  double s = 0.0;
  if (lid < D)
    for (int i = 0; i < K; ++i) s += cabs2(MA[i * D + lid]);
  double t = s * s;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const double nrm = sqrt(t);
  if (lid < D) lam[bond * D + lid] = nrm > 0.0 ? s / nrm : 0.0;
}

// g = 1 (n_g x n_g), the SU metric in the weighted reduced space.
__global__ void k_identity_metric(int ng, double2* g) {
  const size_t nn = (size_t)ng * ng;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn;
       i += (size_t)gridDim.x * blockDim.x)
    g[i] = make_double2((i / ng == i % ng) ? 1.0 : 0.0, 0.0);
}

cudaError_t launch_su_weight(ntu_ctx* c, int skip, int inverse, int normalise,
                             const double2* A, const double2* B, double2* Aout, double2* Bout) {
  const Plan& P = c->plan;
  k_su_weight<<<2, NTU_CTA, 0, c->stream>>>(P.dp, P.D, skip, inverse, normalise, c->w.lam, A, B,
                                            Aout, Bout);
  return after_launch(c, "k_su_weight");
}

cudaError_t launch_su_lambda(ntu_ctx* c, int bond) {
  const Plan& P = c->plan;
  k_su_lambda<<<1, 32, 0, c->stream>>>(P.K, P.D, c->w.MA, c->w.lam, bond);
  return after_launch(c, "k_su_lambda");
}

cudaError_t launch_identity_metric(ntu_ctx* c, double2* g) {
  const Plan& P = c->plan;
  const long long nn = (long long)P.ng * P.ng;
  int blocks = (int)((nn + NTU_CTA - 1) / NTU_CTA);
  if (blocks > 1024) blocks = 1024;
  k_identity_metric<<<blocks, NTU_CTA, 0, c->stream>>>(P.ng, g);
  return after_launch(c, "k_identity_metric");
}

}  // namespace ntu
