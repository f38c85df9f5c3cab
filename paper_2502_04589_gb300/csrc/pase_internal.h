// Internal declarations shared by the translation units of libpase.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/pase.h"

namespace pase {

// ------------------------------------------------------------------ error plumbing
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define PASE_CUDA(call)                                                                 \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::pase::fail(e_ == cudaErrorMemoryAllocation ? PASE_ERR_OUT_OF_MEMORY      \
                                                          : PASE_ERR_CUDA,              \
                          std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

#define PASE_TRY(expr)        \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != PASE_OK) return rc_; \
  } while (0)

// ------------------------------------------------------------------ host CSR
struct HostCSR {
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int64_t nnz() const { return (int64_t)col.size(); }
};

int ensure_max_smem(const void* func, int bytes);
// bracket a launch of kernel `id` with timing events when that kernel is selected
void prof_begin(pase_ctx* h, int id);
void prof_end(pase_ctx* h, int id);
int launch_coldot(pase_ctx* h, int64_t n, int m, const double* X, const double* Y, double* out);
int launch_ratio(pase_ctx* h, int m, const double* num, const double* den, double* out);
int launch_cg_update(pase_ctx* h, int64_t n, int m, const double* alpha, const double* P, const double* Q,
                     double* X, double* R);
int launch_cg_dir(pase_ctx* h, int64_t n, int m, const double* beta, const double* Z, double* P);
int launch_f32_to_f64(pase_ctx* h, int64_t count, const float* x, double* y);
int csr_from_abi(const pase_csr* in, HostCSR& out, const char* name);
HostCSR csr_transpose(const HostCSR& a);
HostCSR csr_multiply(const HostCSR& a, const HostCSR& b);  // a * b
HostCSR csr_galerkin(const HostCSR& P, const HostCSR& A);   // P^T A P
bool same_pattern(const HostCSR& a, const HostCSR& b);
// dense inverse of an SPD CSR matrix (row-major n x n); returns false if not SPD
bool dense_spd_inverse(const HostCSR& a, std::vector<double>& inv);

// ------------------------------------------------------------------ device CSR
struct DevCSR {
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;   // FP64 values
  float* val32 = nullptr;  // FP32 copy (mixed precision), may be null
  int block = 0;           // threads per block of the CSR kernel (0 = 256; set by the autotuner)
  // structured-grid form of the FP32 values (stencil.cu): 3^d tap planes then 1 / a_ii,
  // x extent padded to st_xp; null when the matrix is not a grid-neighbour stencil
  float* st_val = nullptr;
  float* st_jval = nullptr;  // the same for the damped-Jacobi iteration matrix at omega st_omega
  double st_omega = 0.0;
  int st_dim = 0, st_n1 = 0, st_xp = 0;
  // schedule of the FP32 sweeps on this level, set by the autotuner: structured kernel or
  // CSR; resident CTAs per SM of the structured kernel (0 = as many as fit, up to 2); work
  // items per resident CTA (plane chunks of a tile); columns per consumer thread (4, or 2:
  // twice the threads at half the registers)
  int st_use = 1, st_per_sm = 0, st_items = 6, st_cw = 4;
};

struct Level {
  DevCSR A;                  // A_l (level 0: A_h; shares col/rowptr with M)
  double* dinv = nullptr;    // 1 / diag(A_l)
  float* dinv32 = nullptr;
  DevCSR P;                  // interpolation level l+1 -> l  (rows n_l)
  DevCSR PT;                 // its transpose (rows n_{l+1})
};

// Per-block-width workspace.
struct Work {
  int m = 0;
  int64_t N = 0;
  // fine level multivectors [N][m]
  double *R = nullptr, *E = nullptr, *T1 = nullptr, *T2 = nullptr, *W = nullptr, *U = nullptr;
  double* lam = nullptr;                     // [m]
  // per level (l >= 1) multivectors: b, x, t1, t2  [n_l][m]
  std::vector<double*> lb, lx, lt1, lt2;
  // FP32 copies for the mixed-precision solve, all levels (level 0 included)
  std::vector<float*> fb, fx, ft1, ft2;
  // reductions
  double* partial = nullptr;  // scratch for two-stage reductions
  size_t partial_bytes = 0;
  double* norms = nullptr;    // [4m]
  double* relres = nullptr;   // [m]
  // projection outputs
  double *aH = nullptr, *bH = nullptr, *GA = nullptr, *GM = nullptr;
  double *CH = nullptr, *CW = nullptr;
  // augmented eigensolver (n_c = N_H + m rows, up to 3m wide)
  double *S = nullptr, *AS = nullptr, *BS = nullptr;   // [n_c][3m]
  double *Xn = nullptr, *AXn = nullptr, *BXn = nullptr;  // [n_c][m]
  double *Pn = nullptr, *APn = nullptr, *BPn = nullptr;  // [n_c][m]
  double *Gq = nullptr, *Gb = nullptr, *Cs = nullptr;   // small dense [3m][3m], C [3m][m]
  double *ahat = nullptr, *schur = nullptr;             // [N_H][m], [m][m]
  double* eigwork = nullptr;                            // small eigensolver scratch
  size_t eigwork_doubles = 0;
  double* smallvec = nullptr;                           // [16m]
  double *Rn = nullptr, *coef = nullptr;                // [n_c][m], [m][m]
  double *cgP = nullptr, *cgQ = nullptr;                // CG direction and A times it [N][m]
  double* cgs = nullptr;                                // CG scalars: (r,z) x2, (p,Ap), ratio [4m]
  int* status = nullptr;                                // device status words [8]
  int* colexp = nullptr;                                // split Gram column exponents [3][128]
  float *dfh = nullptr, *dfl = nullptr;                 // double-float split of a block [N][m]
  int* df_flag = nullptr;                               // a split value was outside 2^+-100
  // small spaces solved densely: the coarse pencil [N_H][N_H] (filled at reserve) when
  // N_H <= 3m; the augmented pencil [n_c][n_c] and its m smallest eigenvectors [n_c][m]
  // when n_c = N_H + m <= 3m
  bool coarse_dense = false, aug_dense = false;
  double *AHd = nullptr, *MHd = nullptr, *Ad = nullptr, *Bd = nullptr, *Cd = nullptr;
  // step-(c) congruences (aug_transform): Z, the transformed blocks, coarse CG buffers
  double *Zt = nullptr, *aT = nullptr, *bT = nullptr, *GAT = nullptr, *GMT = nullptr;  // [N_H][m], [m][m]
  double *tr = nullptr, *tz = nullptr, *tp = nullptr, *tq = nullptr, *tsc = nullptr;   // [N_H][m] x4, [4m]
  // control block of the device-decided loops (flow.cu): ints [kCtlInts], doubles [CD_COUNT]
  int* ci = nullptr;
  double* cd = nullptr;
  // host pinned mirror for small readbacks
  double* h_small = nullptr;
  int* h_status = nullptr;
  int* h_ci = nullptr;
  double* h_cd = nullptr;
};

// ------------------------------------------------------------------ device control block
// Integer words of Work::ci.  The first CI_EXEC0 words are zeroed at the start of a solve;
// the words from CI_EXEC0 on count executions of conditional graph bodies (one per body).
enum CtlInt {
  CI_ERR = 0,    // pending error: a PASE_ERR_* code, or kCtlErrDfRange
  CI_OUT_CONT,   // outer loop goes on
  CI_OUT_GO,     // this outer pass runs an iteration
  CI_ITER,       // outer iterations done
  CI_CONV,       // pairs at tol after the last test
  CI_POST,       // this pass runs the second linear solve of Alg. 3 (post_solve)
  CI_IN_CONT,    // inner (step-(c)) loop goes on
  CI_IN_GO,      // this inner pass updates the block
  CI_IN_OK,      // the pass's small eigensolve succeeded
  CI_IN_IT,      // inner passes of the current step (c)
  CI_AUG_IT,     // inner passes, summed since the solve began
  CI_HIST_N,     // inner residual history length
  CI_MAXED,      // max_iter reached without convergence
  CI_EXEC0 = 16,
};
enum CtlDbl { CD_WORST = 0, CD_AUG_TOL, CD_IN_WORST, CD_PREV_WORST, CD_FACTOR, CD_HIST = 8, CD_COUNT = 16 };
constexpr int kCtlHist = 8;                       // ring of inner residuals (stagnation test)
constexpr int kCtlSlots = 240;                    // conditional bodies with a counter
constexpr int CI_GUARD0 = CI_EXEC0 + kCtlSlots;  // pass guards of the WHILE nodes, one per slot
constexpr int kCtlInts = CI_GUARD0 + kCtlSlots;
constexpr int kCtlErrDfRange = 1;                 // a double-float split met |x| > 2^100
constexpr int kCapMaxDepth = 8;
// counter slots of the recorded graphs of a handle
constexpr int kSlotStepC = 0, kSlotStart = 16, kSlotSolve = 32, kSlotBatch = 136, kSlotsPerSolve = 104;

// A recorded and instantiated CUDA graph with what is needed to count its kernels.
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> key;  // what the recording depends on
  int slot0 = 0, nslots = 0;  // its counter slots
  int64_t top_kernels = 0;    // kernels outside conditional bodies (run once per launch)
  int64_t nodes_recorded = 0; // kernels recorded, bodies included
};
// State of a recording in progress.
struct Capture {
  GraphRec* rec = nullptr;
  int depth = 0;
  int slot_next = 0, slot_end = 0;
  std::vector<int64_t> child;                   // kernels recorded in nested bodies, per level
  std::vector<std::pair<int, int64_t>> bodies;  // (slot, kernels of that body alone)
};

// learned fine-level smoother (smoother.cu)
struct Smoother {
  int dim = 0, n = 0, n1 = 0, T = 0, P = 0;
  int64_t N = 0;
  bool has_params = false;
  bool rejected = false;  // validation after training found it no better than Jacobi
  int t = 0;              // Adam steps taken
  float* feat = nullptr;                                                             // node feature [N]
  float *params = nullptr, *adam_m = nullptr, *adam_v = nullptr, *peff = nullptr;  // [P]
  float* wt = nullptr;                                                               // transposed layer weights
  double *grad = nullptr, *partial = nullptr, *colpart = nullptr;
  float *act0 = nullptr, *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *y = nullptr, *ga = nullptr, *gb = nullptr;
  double *E = nullptr, *AE = nullptr, *e = nullptr, *r = nullptr;  // [N][8] training blocks
  double* sums = nullptr;                                          // small device scalars
  int* tc_err = nullptr;                                           // tensor-core wait timeout flag
  double* h_sums = nullptr;                                        // pinned mirror
};
int smoother_nparams(int dim);
bool sm_active(const pase_ctx* h);
int sm_set_grid(pase_ctx* h, int dim, int n, const double* logk_host);
int sm_state(pase_ctx* h, float* buf, int64_t count, bool get);
template <typename T>
int sm_apply(pase_ctx* h, int m, const T* R, int64_t ldr, const T* dinv, T* X, int64_t ldx, bool add);
int sm_step(pase_ctx* h, const double* e, const double* r, bool update, float lr, float b1, float b2, float eps,
            double* loss_cols);
int sm_jacobi_loss(pase_ctx* h, const double* e, const double* r, double* loss_cols);
int sm_grad_to_host(pase_ctx* h, double* grad_host);
int sm_check_timeout(pase_ctx* h);  // PASE_ERR_TIMEOUT if a tensor-core wait gave up (then clears it)
void sm_free(pase_ctx* h);

}  // namespace pase

struct pase_ctx {
  pase_options opt;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 152;         // multiprocessors of the device (queried at create)
  int* tc_err = nullptr;     // device flag: a tensor-core wait of the split GEMM ran out
  bool ready = false;
  int L = 0;             // number of levels (chain length + 1)
  int coarse_level = 0;  // which level is V_H
  int64_t N = 0, NH = 0;
  std::vector<pase::Level> lv;
  double* M0_val = nullptr;  // M_h values (pattern of A_h)
  float* M0_val32 = nullptr;
  float *A0h = nullptr, *A0l = nullptr, *M0h = nullptr, *M0l = nullptr;  // double-float split of A_h, M_h
  pase::DevCSR Pd, PdT;      // direct interpolation V_H -> V_h and its transpose
  pase::DevCSR AH;           // coarse pencil as given: A_H with values, M_H values below
  double* MH_val = nullptr;
  double* MH_dinv = nullptr;  // 1 / diag(M_H) (Jacobi-preconditioned CG with the coarse mass)
  int64_t ncoarsest = 0;     // dense inverse of the coarsest multigrid operator
  double* cinv = nullptr;
  float* cinv32 = nullptr;
  pase::Work w;
  int64_t launches = 0;
  int aug_nconv = 0;         // columns the step-(c) solver must converge (0 = all)
  // CUDA graph of the step-(a) linear solve (captured once per handle inside pase_solve)
  cudaGraphExec_t ls_graph = nullptr;
  const double* ls_graph_U = nullptr;
  double* ls_graph_W = nullptr;
  int64_t ls_graph_kernels = 0;
  // live timing of one kernel (pase_profile_kernel): event pairs on the handle's stream
  int prof_kernel = -1;
  std::vector<cudaEvent_t> prof_ev;
  size_t prof_n = 0;
  const double* ls_last_U = nullptr;  // buffers of the previous step-(a) call
  const double* ls_last_W = nullptr;
  bool graphs_ok = true;
  int tuned_m = 0;
  // device staging buffers for host-memory arguments, kept between calls (grow-only;
  // a buffer is busy while the call that took it runs)
  struct StageBuf {
    void* p;
    size_t bytes;
    bool busy;
  };
  std::vector<StageBuf> stage_pool;
  pase::Smoother* sm = nullptr;  // learned smoother (pase_set_grid)
  bool sm_suspend = false;       // Jacobi while the trainer generates samples
  double aug_tol_now = 0;    // current inner tolerance
  // batch scheme (pase_solve_batches): dense coarse pencil and augmented-pencil buffers,
  // allocated on first use (sizes fixed by the first call's nev and m)
  struct BatchBufs {
    int nev = 0, m = 0, top = 0, n = 0, kk = 0, nw = 0;
    double *AHd = nullptr, *MHd = nullptr, *CHc = nullptr, *lamH = nullptr;  // coarse pencil, pairs
    double *Ad = nullptr, *Bd = nullptr, *Cw = nullptr, *lamw = nullptr;    // augmented pencil, pairs
    double *Cc = nullptr, *Rm = nullptr, *Rt = nullptr, *Rt2 = nullptr, *S = nullptr, *comp = nullptr;
    double* eig = nullptr;  // small eigensolver workspace
    size_t eig_doubles = 0;
    int* idx = nullptr;
  } bb;
  std::vector<void*> allocations;
  // recorded graphs (flow.cu): step (c), the coarse start, a whole solve, a solve inside
  // a batch graph; the private streams that recordings capture on
  pase::GraphRec g_stepc{nullptr, {}, pase::kSlotStepC, 16, 0, 0};
  pase::GraphRec g_start{nullptr, {}, pase::kSlotStart, 16, 0, 0};
  pase::GraphRec g_solve{nullptr, {}, pase::kSlotSolve, pase::kSlotsPerSolve, 0, 0};
  pase::GraphRec g_batch{nullptr, {}, pase::kSlotBatch, pase::kSlotsPerSolve, 0, 0};
  pase::Capture cap;
  std::vector<cudaStream_t> cap_streams;
  int64_t body_kernels[pase::kCtlSlots] = {};  // kernels of the body that owns each slot
  int ci_last[pase::kCtlSlots] = {};           // execution counts at the last read
  // tuned small eigensolver per Rayleigh-Ritz size: threads of its single-CTA stages, the
  // tridiagonalisation's form (0 one CTA, 1 a cluster of 8 SMs, 2 of 16) and the Cholesky
  // factorisation's (0 one CTA, 1 a cluster of 8 SMs); -1: by size
  int sygv_n[3] = {0, 0, 0}, sygv_thr[3] = {1024, 1024, 1024}, sygv_cl[3] = {-1, -1, -1}, sygv_ch[3] = {-1, -1, -1};
  int64_t graph_launches = 0;                  // CUDA graph launches issued
  int64_t replayed = 0;                        // kernels (of `launches`) run inside graph replays
  uint64_t serial = 0;                         // unique id of the handle (batch graph keys)
  cudaGraphExec_t batch_exec = nullptr;        // batch graph led by this handle
  std::vector<uint64_t> batch_key;
};

namespace pase {

// ------------------------------------------------------------------ memory helpers
int dev_alloc(pase_ctx* h, void** p, size_t bytes);
template <typename T>
int dev_alloc_t(pase_ctx* h, T** p, size_t count) {
  return dev_alloc(h, (void**)p, count * sizeof(T));
}
int upload_csr(pase_ctx* h, const HostCSR& a, DevCSR& d, bool with_fp32, bool share_pattern_from,
               const DevCSR* src_pattern);

// ------------------------------------------------------------------ sparse kernels
// Modes of the generic CSR x multivector kernel.
enum CsrMode {
  CSR_MV = 0,       // Y1 = A X
  CSR_MV_AM = 1,    // Y1 = A X, Y2 = M X (shared pattern, second value array vm)
  CSR_RESID = 2,    // Y1 = B - A X
  CSR_MVDOT = 7,    // Y1 = A X and per-block column sums of X .* (A X) (square A)
  CSR_JACOBI = 3,   // Y1 = X + omega dinv (B - A X)
  CSR_EIGRES = 4,   // Y1 = (M X) diag(lam) - A X, partial column sums of |Y1|^2, |MX|^2
  CSR_MV2 = 5,      // Y1 = A X, Y2 = A X2 (two inputs, one matrix)
  CSR_ADD = 6,      // Y1 = B + A X
};

template <typename T>
int launch_csr(pase_ctx* h, int mode, int m, const DevCSR& A, const T* va, const T* vm,
               const T* X, const T* X2, const T* B, const T* dinv, const double* lam, double omega,
               T* Y1, T* Y2, double* partial, int* nblocks_out, int64_t ldx = 0,
               int64_t ldy = 0);

// double-float products of the fine level (df64.cu)
int launch_split_df64(pase_ctx* h, int64_t count, const double* x, float* hi, float* lo, int* flag);
int launch_csr_df64(pase_ctx* h, int mode, int m, const DevCSR& A, const float* ah, const float* al,
                    const float* mh, const float* ml, const float* xh, const float* xl, const double* lam,
                    double* Y1, double* Y2, double* partial, int* nblocks_out);

// structured-grid FP32 kernels (stencil.cu)
int stencil_setup(pase_ctx* h, const HostCSR& A, const std::vector<double>& dinv, DevCSR& d);
bool stencil_ok(const DevCSR& A, int mode, int m, int64_t ldx, int64_t ldy, double omega);
int launch_stencil(pase_ctx* h, int mode, int m, const DevCSR& A, const float* X, const float* B, double omega,
                   float* Y);

// elementwise
template <typename T>
int launch_scale_dinv(pase_ctx* h, int64_t n, int m, const T* dinv, double omega, const T* B,
                      T* Y);  // Y = omega dinv B
int launch_axpy(pase_ctx* h, int64_t count, double a, const double* x, const double* y,
                double* z);  // z = a x + y
int launch_f64_to_f32(pase_ctx* h, int64_t count, const double* x, float* y);
int launch_add_f32_to_f64(pase_ctx* h, int64_t count, const double* u, const float* e,
                          double* w);  // w = u + e
int launch_copy_cols(pase_ctx* h, int64_t n, int k, const double* src, int lds, double* dst,
                     int ldd);
int launch_fill(pase_ctx* h, int64_t count, double v, double* x);
int launch_zero_cols_if(pase_ctx* h, int64_t n, int m, int64_t ld, const double* crit, double thresh,
                        double* X, const double* thresh_dev = nullptr);  // thresh_dev: read instead
int launch_hash_fill(pase_ctx* h, int64_t rows, int cols, int64_t ld, unsigned seed, double* X);
int launch_set_identity_rows(pase_ctx* h, int64_t row0, int k, int64_t ld, double* X);
int launch_geam(pase_ctx* h, int64_t rows, int cols, double a, const double* A, int64_t lda,
                double b, const double* B, int64_t ldb, double* C, int64_t ldc);  // C = aA + bB

// reductions
int launch_reduce_partials(pase_ctx* h, int nblk, int width, const double* partial,
                           double* out);  // out[j] = sum_b partial[b*width + j]
int launch_relres(pase_ctx* h, int m, const double* norms, const double* lam, double* relres);

// dense tall-skinny
int ts_gram(pase_ctx* h, int64_t n, int k1, int k2, const double* X, int ldx, const double* Y,
            int ldy, double* G, int ldg, bool sym);  // G = X^T Y (k1 x k2)
// Y = X C on the BF16 tensor cores with FP64 accuracy (split_gemm.cu); k1, k2 even <= 128,
// 16-byte aligned rows.  err: device flag set if a tensor-core wait runs out.
bool ts_gemm_split_ok(int k1, int k2, const void* X, int64_t ldx, const void* Y, int64_t ldy);
int ts_gemm_split(pase_ctx* h, int64_t n, int k1, int k2, const double* X, int64_t ldx, const double* C, int ldc,
                  double* Y, int64_t ldy, int* err);
// GA = W^T Y1, GB = W^T Y2 (upper triangles mirrored), [n][m] blocks with m <= 128 even,
// on the tensor cores with the same splitting (split_gemm.cu); colexp: 3 x 128 ints.
bool ts_gram2_split_ok(int64_t n, int m, int num_sms, const Work& w);  // shape and scratch fit
int ts_gram2_split(pase_ctx* h, int64_t n, int m, const double* W, const double* Y1, const double* Y2, double* GA,
                   double* GB, int ldg, int* colexp, int* err);
int ts_gemm(pase_ctx* h, int64_t n, int k1, int k2, double alpha, const double* X, int ldx,
            const double* C, int ldc, double beta, double* Y, int ldy);  // Y = a X C + b Y
template <typename T>
int dense_mm(pase_ctx* h, int64_t n, int m, const T* Ainv, const T* B, T* X);  // X = Ainv B

// dense helpers of the batch scheme: CSR rows into a dense block, transpose, column gather
int launch_csr_to_dense(pase_ctx* h, int64_t n, int64_t ncols, const int64_t* rowptr, const int32_t* col,
                        const double* val, double* D, int64_t ld);
int launch_transpose(pase_ctx* h, int64_t rows, int64_t cols, const double* A, int64_t lda, double* B, int64_t ldb);
int launch_gather_cols(pase_ctx* h, int64_t n, int k, const double* src, int64_t lds, const int* idx, double* dst,
                       int64_t ldd);

// small dense matrices on one CTA
// smallest Rayleigh-Ritz size the autotuner tries the 16-SM cluster tridiagonalisation on
constexpr int kTri16Min = 96;
int small_sygv(pase_ctx* h, int n, int k, const double* GA, int lda, const double* GB, int ldb,
               double* lam, double* C, int ldc, int* status_dev);
int small_gemm(pase_ctx* h, int m, int n, int k, double alpha, const double* A, int lda,
               bool transA, const double* B, int ldb, double beta, double* C, int ldc);
int small_chol_solve(pase_ctx* h, int n, int nrhs, double* S, int lds, double* B, int ldb,
                     int* status_dev, bool factor);  // [S <- chol(S) (lower)], B <- S^-1 B
size_t small_sygv_work_doubles(int n, int k);
// Cap on the grid of every kernel that writes per-block partial sums (the residual, the
// CG inner products, the smoother's column sums): partial buffers hold this many blocks.
constexpr int kReduceBlocksHost = 152 * 8;
// FP64 FMA-rate launch (pase_time_kernel PASE_KERNEL_FMA_FP64): 2 * 8 * iters * threads * blocks flops
constexpr int kFmaBlocks = 152 * 8, kFmaThreads = 256, kFmaIters = 4096;
int launch_fma_fp64(pase_ctx* h, double* out);
// device-decided control flow (flow.cu)
bool recording(const pase_ctx* h);
// A conditional node at the current point of the recording: IF (loop false) runs body once
// when *flag != 0; WHILE runs it while *flag != 0 after each pass, at most max_passes
// passes (then PASE_ERR_TIMEOUT in the control block).
int cond_node(pase_ctx* h, bool loop, int* flag, const std::function<int()>& body, int max_passes = 0);
int graph_record(pase_ctx* h, GraphRec& rec, const std::function<int()>& fn);
int batch_record(pase_ctx* const* hs, int count, const std::function<int(int)>& fn, cudaGraphExec_t* out);
int graph_launch(pase_ctx* h, GraphRec& rec);
void graph_free(GraphRec& rec);
int sync_ctl(pase_ctx* h, const double* src = nullptr, int count = 0);
int launch_ctl_init(pase_ctx* h);
int launch_ctl_put(pase_ctx* h, int* pi, int vi, bool add, double* pd, double vd);
int launch_ctl_outer_check(pase_ctx* h, int nev, double tol);
int launch_ctl_aug_tol(pase_ctx* h, int nev);
int launch_ctl_inner_init(pase_ctx* h);
int launch_ctl_inner_check(pase_ctx* h, int nconv, const double* relres, const double* tol_dev, double tol_fixed,
                           int maxit);
int launch_ctl_status(pase_ctx* h, const int* status, bool fatal);
// column-wise residual of a block eigenproblem: R = AX - BX diag(lam), partial norms
int launch_block_resid(pase_ctx* h, int64_t n, int m, const double* AX, const double* BX,
                       int64_t ldin, const double* lam, double* R, int64_t ldr, int* nblk_out);

}  // namespace pase
