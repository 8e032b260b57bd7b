// Shared-memory layout and launch arguments of the ALS kernel k_als
// (als_kernel.cuh), and the launchers of its instantiations, one per
// translation unit: the lane build of the reduced metric only, and the
// tensor-core build at K = 16 and at K = 32.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "ntu_dev.cuh"
#include "ntu_impl.h"
#include "oz_build.cuh"

namespace ntu {

// The members keep fixed offsets from the dynamic shared-memory base, so
// that every access is a constant address.  The SVD work arrays S come last:
// the tensor-core build carves its 1024-byte aligned pieces from S, which
// may run up to ALS_OZ_SLACK bytes past its end (the launch adds them).
struct AlsShared {
  double2 MA[32 * 8];
  double2 MB[32 * 8];
  double2 y[256];
  double2 y2[256];
  double2 p[256];
  double2 ap[256];
  double2 ph[32];
  int ge;                      // scale exponent of the double-FP32 copy of g
  double red[2 * NTU_WARPS];
  double eps0, tau_sel;
  int err;
  int flag;
  int n_cg, n_fast, n_eig;
  SvdSmem S;
};
constexpr size_t ALS_OZ_SLACK = 1024;
static_assert(offsetof(AlsShared, S) + sizeof(SvdSmem) == sizeof(AlsShared),
              "the SVD work arrays end the ALS shared memory");
static_assert(OZ_SMEM_BYTES + 1023 <= sizeof(SvdSmem) + ALS_OZ_SLACK,
              "the tensor-core build fits in the SVD work arrays and the slack after them");

struct AlsArgs {
  int D, K, ng, nA, sweeps, kmin, kmax;
  const double2* g; const double2* RA; const double2* RB;
  double2* MA; double2* MB; double* info;
  int* path_counts;            // [Gershgorin+CG, shifted Cholesky, eigen] solves (may be NULL)
  double2 *x0, *gx0, *Tm, *gA, *gC, *jv, *pv, *tauv;
  double *dv, *ev, *rc, *rs;
  int* rk;
  int rotcap;
  int* status;
  int df;                      // build the reduced metric in double-FP32 arithmetic
  float4* gdf;                 // n x ng^2: g 2^-e split into FP32 pairs (k_gsplit)
  float4* gdfT;                // the same with kA and kB swapped in rows and columns
                               // (written for the lane build only)
  int split;                   // CTAs per item (a cluster); the private scratch above
                               // (x0 ... rk, gA, gC) has n * split copies
  int* sync;                   // n exchange counters, zero at launch (split > 1)
  long long wait_polls;        // poll limit of a rendezvous
  int sync_extra;              // 0; 1 only under ntu_inject_wait_timeout
  int oz;                      // build the first stage on the tensor cores (K = 16)
  __nv_bfloat16* gsl;          // n x 2 x rows_side x 64 slices of g (oz_build.cuh)
  short* gexp;                 // n x 2 x K x n_g exponents of the slice segments
  const int* gscale;           // n scale exponents e of the double-FP32 g (k_gsplit)
  const CUtensorMap* gmap;     // TMA map of gsl, in global memory (a tensor map as a
                               // kernel parameter slowed this kernel down 1.85x)
};

// Launch n items of the ALS on `split` CTAs each (a cluster for split > 1);
// `three`: the three-CTAs-per-SM register budget (split 1 only).  Return the
// launch error.
cudaError_t als_launch_lanes(const AlsArgs& a, int n, int split, bool three, size_t smem,
                             cudaStream_t stream);
cudaError_t als_launch_tc16(const AlsArgs& a, int n, int split, bool three, size_t smem,
                            cudaStream_t stream);
cudaError_t als_launch_tc32(const AlsArgs& a, int n, int split, bool three, size_t smem,
                            cudaStream_t stream);

}  // namespace ntu
