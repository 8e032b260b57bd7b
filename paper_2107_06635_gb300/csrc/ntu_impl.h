// Internal declarations of the NTU library: the per-configuration plan
// (sizes and contraction index tables), the device work space and the
// kernel launchers that the C ABI (capi.cu) strings together.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ntu.h"

namespace ntu {

// One batched complex GEMM of the environment contraction (Fig. 4):
//   C[b][rowC[m] + colC[n]] = sum_k A[b][rowA[m] + kA[k]] * B[b][kB[k] + colB[n]]
// with optional conjugation of A or B.  The six index tables map the
// composite tensor indices to element offsets; they live in one device int
// array at the given offsets.  mode 1 / 2 / 3 (FP32 path only) write the
// result instead as the split-BF16 operand of a tensor-core GEMM (see
// k_tc.cu): row rowC[m] + colC[n], complex column rowK[m] + colK[n], row
// pitch `pitch` BF16 elements, lo half at +krp_out; mode 2 doubles the rows;
// mode 3 doubles them with Re / Im factors planar in K (krp_out / 2 apart).
struct GemmOp {
  int M, N, Kd;
  int rowA, kA, kB, colB, rowC, colC;   // offsets into the table array
  int conjA, conjB;
  long long sA, sB, sC;                 // per-item strides (elements of the output)
  int mode, rowK, colK, pitch, krp_out;
};

// Arguments of one tensor-core GEMM (k_tc.cu) as seen by the kernel.
struct TcArgs {
  int kTiles;            // 64-wide K tiles per split pass
  int krp;               // padded real K of one half ([hi | lo] rows are 2 krp wide)
  int Mc, N;             // valid complex rows, valid columns
  int mtiles;            // 128-row tiles of the doubled A operand
  const int *rowC, *colC, *rowK, *colK;
  void* out;
  long long sOut;        // per-item stride of the output (elements)
  int pitch, krp_out;    // split outputs: row pitch and lo offset (BF16 elements)
  int vec4;              // split outputs: groups of four columns are consecutive in one row
  int* err;
};

// A tensor-core GEMM of the plan: operand tensor maps, kernel arguments,
// table offsets and output mode (0 complex FP32, 1 split operand, 2 split
// doubled operand).
struct TcOp {
  CUtensorMap mapA, mapB;
  TcArgs args;
  int rowC, colC, rowK, colK;
  int mode, mtiles;
};

struct Plan {
  int D, d, d_anc, dp, r, K, m, ng, nA;
  long long szT, szQ, szR, szE1, szE2, szS2, szG;
  GemmOp eL, eR, eTL, eBL, eTR, eBR;    // edge double tensors (Fig. 4(b))
  GemmOp y, t1, t2, h;                  // half environment steps (Fig. 4(c,d))
  GemmOp join;                          // join of the two halves (Fig. 4(d,e))
  // split-BF16 tensor-core variant (NTU_MIXED_BF16X3)
  GemmOp e2TL, e2BL, e2TR, e2BR;        // edge tensors written as doubled A operands
  TcOp tc_hL, tc_hR, tc_join;
  long long krpY, rowsY, rowsQ;         // split operands of the fused t1-t2: Y (doubled A), conj(Q) (B)
  CUtensorMap mapYs, mapQs;             // TMA maps of the fused t1-t2 (k_t12.cu)
  CUtensorMap mapT2st;                            // its output T2s, box D^2 rows (TMA store)
  long long krpE, krpJ;                 // padded real K of the t2/h and join GEMMs
  long long rowsE, rowsT, rowsHL, rowsHR;  // allocated rows of the split operands
  int* d_tab;                           // device index tables
  int n_tab;
  // tensor-core build of the ALS reduced metric (K = 16, mixed contexts)
  int oz_ok;
  CUtensorMap mapGsl;                   // slices of g, box 128 rows x 64 BF16
};

// Device work space for max_batch items.  Every pointer is the base of a
// stack of per-item slices.
struct Work {
  int cap;               // items
  double2 *GA, *GB;      // split gate halves, d*d*r each
  double2 *Mg, *Qcm;     // gated matrices / Q scratch, 2 * m*K each (both sides)
  double2 *QA, *QB, *RA, *RB;
  // environment (element type: double2 for FP64, float2 for the mixed paths)
  void *Tac, *Tbc, *QAc, *QBc, *EL, *ER, *ETL, *EBL, *ETR, *EBR, *Y, *T1, *T2, *HL, *HR, *graw;
  // split-BF16 operands of the tensor-core environment
  void *ETLd, *EBLd, *ETRd, *EBRd, *T2s, *HLd, *HRs, *Ys, *Qs;
  int* qrflag;           // 2 per item: QR left to the Householder kernel
  double2 *g, *gscr, *gw;     // metric, Cholesky / eigen scratch, eigenvectors
  double *gz, *geig;          // explicit Z (ng*ng) and d,e (2*ng) for the repair fallback
  double2 *gtau, *gp;         // reflector factors, vector scratch (ng each)
  double *diag;               // 3 per item
  // ALS scratch
  // (private per CTA: cap x als_split copies, see k_als)
  double2 *x0, *gx0, *Tm, *gA, *gC, *jv, *pv, *tauv;
  double *dv, *ev, *rc, *rs;
  int *rk;
  int rotcap;
  int als_split;              // most CTAs one item's ALS may use (1, 2 or 4)
  int* als_sync;              // cap exchange counters of the split ALS
  unsigned long long* gmaxb;  // cap: largest |entry| of each item's g (bit pattern)
  int* gscale;                // cap: scale exponent e of each item's double-FP32 g
  double2 *MA, *MB;
  double *info;               // 4 per item
  // outputs of a full update when the caller gives none
  double2 *Ta_out, *Tb_out;
  // inputs staged for host-pointer calls
  double2 *Ta_in, *Tb_in, *G_in;
  // unit cell of the context
  double2 *A, *B, *cTa, *cTb, *cG, *op;
  double2 *cA2, *cB2;
  double2 *mscr1, *mscr2, *medge;   // measurement scratch
  double2 *mval;
  double* lam;                // simple update: bond tensors lambda_0..3 (4 x D)
  void* gsl;                  // tensor-core ALS build: BF16 slices of g (n x 3 MB at K = 16)
  short* gexp;                // and their exponents
  CUtensorMap* gmap;          // the TMA map of gsl, copied to device memory
};

}  // namespace ntu

struct ntu_ctx {
  ntu_config cfg;
  cudaStream_t stream;
  bool own_stream;
  ntu::Plan plan;
  ntu::Work w;
  int* d_status;
  char err[320];
  int launches;
  int stage;          // 0 none, 1 after apply_gate, 2 after env_metric
  int stage_bond;
  size_t env_es;      // element size of the environment buffers
  int profiling;
  cudaEvent_t ev[6];
  cudaStream_t copy_stream;   // host-buffer batches: the overlapped copies (created on use)
  cudaEvent_t cev[3];
  int* d_paths;       // [ALS Gershgorin+CG, ALS shifted Cholesky, ALS eigen,
                      //  repair Gershgorin, repair Cholesky, repair eigen,
                      //  QR CholeskyQR2, QR Householder]
  int debug_sync;     // synchronise and check after every launch (NTU_DEBUG_SYNC=1)
  int sms;            // streaming multiprocessors of the context's device
  long long wait_polls;   // poll limit of the ALS rendezvous (wait_budget, or 2^23)
  int inject_timeout;     // ntu_inject_wait_timeout: rendezvous target one too high
  ntu_tuning tune;        // schedule choices (ntu_set_tuning)
  int use_graphs;         // capture the unit-cell step as a CUDA graph
  cudaGraphExec_t step_graph[4];  // [ntu_step, ntu_su_step] x [no gate1, gate1]
  int step_graph_launches[4];
};

namespace ntu {

// drop the captured unit-cell step graphs (after a change that they bake in)
void drop_step_graphs(ntu_ctx* c);
// error helper: record message, return status
int fail(ntu_ctx* c, int status, const char* fmt, ...);
// Called after every launch: counts it and, in debug mode, synchronises and
// reports the first failing kernel by name.
cudaError_t after_launch(ntu_ctx* c, const char* name);

// plans and tables (k_env.cu)
int plan_build(ntu_ctx* c);
int init_context(const ntu_config* cfg, void* stream, ntu_ctx** out, int max_split);
void plan_free(ntu_ctx* c);

// launchers (return cudaError_t of the launch; they also count launches)
cudaError_t launch_gate_qr(ntu_ctx* c, int n, const double2* Ta, const double2* Tb,
                           const double2* G, int swap_sites, double2* QA, double2* RA,
                           double2* QB, double2* RB);
cudaError_t launch_env(ntu_ctx* c, int n, const double2* Ta, const double2* Tb,
                       const double2* QA, const double2* QB, void* graw);
cudaError_t launch_repair(ntu_ctx* c, int n, const void* graw, int raw_is_f32, double2* g,
                          double* diag);
// sweeps < 0: the context's als_sweeps
cudaError_t launch_als(ntu_ctx* c, int n, const double2* g, const double2* RA,
                       const double2* RB, double2* MA, double2* MB, double* info,
                       int sweeps = -1);
cudaError_t launch_recompose(ntu_ctx* c, int n, const double2* QA, const double2* QB,
                             const double2* MA, const double2* MB, double2* Ta_out,
                             double2* Tb_out);
cudaError_t launch_orient(ntu_ctx* c, int bond, const double2* A, const double2* B,
                          double2* Ta, double2* Tb);
cudaError_t launch_deorient(ntu_ctx* c, int bond, const double2* Ta, const double2* Tb,
                            double2* A, double2* B);
cudaError_t launch_site_gate(ntu_ctx* c, double2* A, double2* B, const double2* op);
cudaError_t launch_measure(ntu_ctx* c, const double2* T, const double2* N, const double2* op,
                           double2* out);
cudaError_t launch_copy_raw(ntu_ctx* c, int n, const void* graw, double2* g);
// simple update (k_su.cu)
cudaError_t launch_su_weight(ntu_ctx* c, int skip, int inverse, int normalise,
                             const double2* A, const double2* B, double2* Aout, double2* Bout);
cudaError_t launch_su_lambda(ntu_ctx* c, int bond);
cudaError_t launch_identity_metric(ntu_ctx* c, double2* g);
size_t als_smem_bytes();
// Box rows of one ALS step's slices of g for the tensor-core build at this
// K (0 where that build does not exist) (k_solve.cu).
long long oz_rows_side(int K);
// Dynamic shared-memory limits of the fixed-size kernels, set on the
// current device when a context is created there (k_gate_qr.cu, k_t12.cu,
// k_tc.cu).
cudaError_t gate_qr_attributes();
cudaError_t t12_attributes();
cudaError_t tc_attributes();

// tensor-core environment (k_tc.cu, k_env.cu)
int tc_make_map(CUtensorMap* map, void* base, long long cols, long long rows, long long items,
                int box_rows = 128);
cudaError_t launch_t12(ntu_ctx* c, int n, const void* Etop);
int tc_plan_maps(ntu_ctx* c);
cudaError_t launch_tc_gemm(ntu_ctx* c, const TcOp& op, int n, void* out);

}  // namespace ntu
