// Gate split + gate application + QR of one bond without any device
// allocation.
//
// Some callers cannot call cudaMalloc: a host framework that owns all device
// memory through its own pool and forbids other allocators, code that must
// not trigger the implicit device synchronisation of cudaMalloc/cudaFree
// (latency-critical loops sharing the GPU with other streams), or callers
// that run where creating an ntu_ctx (which allocates its work space) is
// not possible.  For them, ntu_gate_qr_noalloc runs the same three kernels
// as the context path (k_gate_split, k_gated, k_qr), with their scratch --
// the split gate halves, the two gated site matrices and the Q work buffers
// -- placed in one fixed, file-scope device array instead of the context's
// work space.  The caller still passes inputs and outputs.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "ntu_dev.cuh"
#include "ntu_impl.h"

namespace ntu {
__global__ void k_gate_split(int d, int r, int swap_sites, const double2* G, double2* GA,
                             double2* GB);
__global__ void k_gated(int d, int danc, int D, int r, const double2* Ta, const double2* Tb,
                        const double2* GA, const double2* GB, double2* Mg);
__global__ void k_qr(int m, int K, double2* Mg, double2* Qcm, double2* QA, double2* RA,
                     double2* QB, double2* RB, const int* only, int* paths);
}  // namespace ntu

// 4 MiB of scratch, held by every GPU that loads the library until the
// process exits.  Enough for every configuration with
// 16 * (2 d^2 r + 4 (d_p D^3) (D r)) <= 4 MiB, e.g. D=8, d=2, r=4.
#define NTU_NOALLOC_SCRATCH_BYTES (4u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[NTU_NOALLOC_SCRATCH_BYTES];

// Host copies of the array's device address, one per device.  In host code
// the symbol g_noalloc_scratch is only a host-side stand-in, never a device
// address, so the address is looked up with cudaGetSymbolAddress.  The set-up
// also sets k_gate_split's shared-memory limit on that device, once.  The
// cache assumes the device's context lives as long as the process: after a
// cudaDeviceReset the array may move, so no reset may come between calls.
#define NTU_NOALLOC_MAX_DEVICES 64
static void* g_noalloc_ptr[NTU_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;
static size_t gate_split_smem_bytes() { return sizeof(ntu::SvdSmem) + 16 * 16 * sizeof(double2); }

static int noalloc_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ntu::fail(nullptr, NTU_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= NTU_NOALLOC_MAX_DEVICES)
    return ntu::fail(nullptr, NTU_EUNSUPPORTED, "device %d beyond the %d supported", dev,
                     NTU_NOALLOC_MAX_DEVICES);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return ntu::fail(nullptr, NTU_ECUDA, "cudaGetSymbolAddress of the scratch array: %s",
                       cudaGetErrorString(e));
    e = cudaFuncSetAttribute(ntu::k_gate_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gate_split_smem_bytes());
    if (e != cudaSuccess)
      return ntu::fail(nullptr, NTU_ECUDA, "shared-memory limit of k_gate_split: %s",
                       cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return NTU_OK;
}

extern "C" int ntu_gate_qr_noalloc(int D, int d_phys, int d_anc, int r, const double* Ta,
                                   const double* Tb, const double* gate, double* QA, double* RA,
                                   double* QB, double* RB, void* stream) {
  using namespace ntu;
  if (!Ta || !Tb || !gate || !QA || !RA || !QB || !RB)
    return fail(nullptr, NTU_EINVAL, "ntu_gate_qr_noalloc: NULL argument");
  if (D < 1 || D > 8 || d_phys < 2 || d_phys > 4 || d_anc < 1 || d_anc > 4 || r < 1 ||
      r > d_phys * d_phys || D * r > 32 || d_phys * d_anc * D * D < r)
    return fail(nullptr, NTU_EINVAL, "ntu_gate_qr_noalloc: unsupported D=%d d=%d d_anc=%d r=%d",
                D, d_phys, d_anc, r);
  const size_t dp = (size_t)d_phys * d_anc, K = (size_t)D * r;
  const size_t m = dp * D * D * D;
  const size_t n_gate = (size_t)d_phys * d_phys * r;
  const size_t need = sizeof(double2) * (2 * n_gate + 4 * m * K);
  if (need > NTU_NOALLOC_SCRATCH_BYTES)
    return fail(nullptr, NTU_EINVAL,
                "ntu_gate_qr_noalloc: D=%d d=%d d_anc=%d r=%d needs %zu bytes of scratch, more "
                "than the fixed %u-byte array",
                D, d_phys, d_anc, r, need, NTU_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  int st = noalloc_scratch(&base);
  if (st != NTU_OK) return st;
  double2* GA = (double2*)base;
  double2* GB = GA + n_gate;
  double2* Mg = GB + n_gate;              // 2 m K: gated matrices of both sides
  double2* Qcm = Mg + 2 * m * K;          // 2 m K: Q work buffers of both sides
  cudaStream_t s = (cudaStream_t)stream;
  const size_t sm = gate_split_smem_bytes();
  k_gate_split<<<1, NTU_CTA, sm, s>>>(d_phys, r, 0, (const double2*)gate, GA, GB);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    int zsplit = (int)((m * K + NTU_CTA * 8 - 1) / (NTU_CTA * 8));
    if (zsplit < 1) zsplit = 1;
    k_gated<<<dim3(1, 2, zsplit), NTU_CTA, 0, s>>>(d_phys, d_anc, D, r, (const double2*)Ta,
                                                   (const double2*)Tb, GA, GB, Mg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_qr<<<dim3(1, 2), NTU_CTA, 0, s>>>((int)m, (int)K, Mg, Qcm, (double2*)QA, (double2*)RA,
                                        (double2*)QB, (double2*)RB, nullptr, nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return fail(nullptr, NTU_ECUDA, "ntu_gate_qr_noalloc: %s", cudaGetErrorString(e));
  return NTU_OK;
}
