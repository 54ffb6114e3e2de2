// Internal declarations of the HALLaR sm_103a library: the problem layout in
// HBM, the handle, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hallar.h"

namespace hallar {

// ---------------------------------------------------------------------------
// layout of a problem on the device
// ---------------------------------------------------------------------------
// The merged CSR holds, per row i, the off-diagonal entries of C and of the
// constraint matrices (the merged support S of eq. support S ell and its
// mirror, Section 4).  Per entry: the column (int32), for families with a
// sparse C its value, and for pair families a constraint code:
//   code >= 0        constraint l = code, this entry is the owner (the pair's
//                    first index is this row); it writes r_l.
//   code in [-m, -1] constraint l = -code - 1, mirrored entry.
//   code == kNoCons  a pure C entry (value in cval).
// The diagonal of C plus C_I sits in cdiag[n].
enum Family : int { FAM_DIAG = 0, FAM_EDGE = 1, FAM_EDGE_C = 2 };
constexpr int32_t kNoCons = INT32_MIN;

struct Problem {
  int fam = FAM_DIAG;       // kernel family
  int api_family = 0;       // hallar_family as created
  int64_t n = 0, n1 = 0, m = 0, m_pairs = 0, nnz = 0;
  int has_trace = 0;
  double C_J = 0.0, C_I = 0.0, tau2 = 1.0;
  double b_norm1 = 0.0, c_norm1 = 0.0;
  int* rowptr = nullptr;    // [n+1]
  int* col = nullptr;       // [nnz]
  int* code = nullptr;      // [nnz] (pair families)
  double* cval = nullptr;   // [nnz] (families with sparse C)
  float* cval32 = nullptr;  // float copy for the mixed form
  double* cdiag = nullptr;  // [n]
  double* b = nullptr;      // [m]
  float* cdiag32 = nullptr; // float copies for the mixed form
  float* b32 = nullptr;
};

// the merged problem on the host, before upload (also the building block of
// a batch: one per stacked instance)
struct HostProblem {
  int fam = FAM_DIAG;
  int api_family = 0;
  int64_t n = 0, n1 = 0, m = 0, m_pairs = 0, nnz = 0;
  int has_trace = 0;
  double C_J = 0.0, C_I = 0.0, tau2 = 1.0;
  double b_norm1 = 0.0, c_norm1 = 0.0;
  std::vector<int32_t> rowptr, col, code;
  std::vector<double> val, cdiag, b;
};
// validate and merge (throws Err); see hallar_create for the arguments
void merge_problem(HostProblem& P, int64_t n, int64_t n1, const int64_t* rp, const int32_t* ci,
                   const double* cv, double C_J, double C_I, int family, int64_t m_pairs,
                   const int32_t* pi, const int32_t* pj, int has_trace, const double* b,
                   double tau2);

// ---------------------------------------------------------------------------
// reductions: per-block partials, summed by the last block in a fixed order
// ---------------------------------------------------------------------------
constexpr int kMaxRed = 16;      // scalars per grid reduction
constexpr int kMaxBlocks = 4096; // largest reduction grid
constexpr int kColsumMax = 256;  // column-sum buffers hold up to 256 columns

struct RedBuf {
  double* partials = nullptr;   // [kMaxBlocks * (2 kColsumMax + 2)]
  unsigned* counter = nullptr;
};

// bytes of one timed kernel launch (see op_bytes in kernels_ops.cu): alg with
// the factor's r columns, pad with its stored leading dimension
struct OpBytes {
  double alg = 0.0, pad = 0.0;
};

// ---------------------------------------------------------------------------
// arguments of the operator kernels that the device-side ADAP-AIPP loop
// (loop.cu) rewrites between launches; an entry point passes them by value
// ---------------------------------------------------------------------------
// epilogue of the fused operator (kernels_ops.cu)
enum GradEpi : int { EPI_W = 0, EPI_FISTA_Z = 1, EPI_AIPP = 2 };
struct GradInd {
  const void* U = nullptr;     // factor in
  void* out = nullptr;         // W (EPI_W, may be null) or z (EPI_FISTA_Z)
  void* resid = nullptr;       // residuals out (factor type), or null
  const void* ctr = nullptr;   // prox centre (EPI_FISTA_Z, EPI_AIPP)
  const void* zin = nullptr;   // unprojected step of the accepted y (EPI_AIPP)
  double beta = 0.0, c2lam = 0.0, invL = 0.0, L = 0.0;
  int active = 1, pad = 0;
};
struct VcInd {                 // value change g(Y) - g(X)
  const void* X = nullptr;
  const void* Y = nullptr;     // Y, or Z when Y = cs Z (ADAP-FISTA trial)
  const void* rX = nullptr;    // residuals at X (factor type)
  void* rY = nullptr;          // residuals at Y out, or null
  const void* ctr = nullptr;   // prox centre (Y = cs Z form)
  void* y_out = nullptr;       // Y = cs Z out (Y = cs Z form)
  int active = 1, pad = 0;
};
struct ColInd {                // column-sum pre-passes
  const void* U = nullptr;     // factor (mode 0) or X (mode 1)
  const void* Y = nullptr;     // mode 1: Y, or Z when y_from_z
  int active = 1, y_from_z = 0;
};
struct TraceInd {              // trace-row residual entry
  void* dst = nullptr;
  int active = 1, pad = 0;
};
struct XInd {                  // ADAP-FISTA x and x~ updates
  void* x = nullptr;           // x out
  const void* x_src = nullptr; // x in (the centre on the first update)
  void* xt = nullptr;          // x~ out
  const void* xt_src = nullptr;// x~ in (mode 1)
  const void* y = nullptr;
  double c0 = 0.0, c1 = 0.0, c2 = 0.0, w0 = 0.0, w1 = 0.0;
  int mode = 0, active = 0;    // mode 0: x~ = w0 y + w1 x; mode 1: step 3's x
                               // update, then x~ = w0 y + w1 x
};

// Device-resident state of one ADAP-AIPP call (Appendix A) and of its
// ADAP-FISTA calls (Appendix A.1).  The host fills the fixed part and the
// evolving part's start values, launches the loop (as a CUDA graph of two
// nested WHILE nodes, or kernel by kernel), and reads the results back.
// Factor buffers rotate by index: pool[i_ctr] is the prox centre, pool[i_y]
// the current ADAP-FISTA y and pool[i_ynew] the trial's y; x, x~ and z have
// buffers of their own (x and x~ are the centre until first written).
struct LoopCtl {
  void* pool[3];
  void* xb;
  void* xtb;
  void* zb;
  void* rpool[2];              // residuals at the centre / at the accepted y
  void* rX;                    // residuals at x~
  int i_ctr, i_y, i_ynew, i_rctr;
  int x_alias, xt_alias, mixed, has_trace;
  // fixed for the call
  double beta, tau, chi, sigma, mu, slack_u, rho, C_J, b_tr, p_tr;
  int max_fista, max_aipp, attempt_cap, trial_cap;
  // evolving
  double lam, Mbar, nrm_ctr2;
  double A, tk, L, Ln, a, Lacc;
  int fista_it, fista_status, trials, aipp_j;
  int done, attempts, error, graph_mode;
  int stall_exit;              // done on a prox step that left W unchanged
  int verbose;                 // >= 3: the control kernels print their step-2 tests
  // operator scalars at the accepted W (valid when done)
  double gT0, gpr, grr, gmag, gnrm2, gWU, Rn;
  // counters since the call started
  long long n_fista_iters, n_fista_fail, n_aipp_iters, n_grads, n_values, n_trials, n_attempts;
  unsigned long long h_fista, h_aipp;  // cudaGraphConditionalHandle of the two loops
  int cont_fista, cont_aipp;           // loop conditions (read by the host in kernel-by-kernel mode)
  // kernel argument blocks
  GradInd g_trial, g_check;
  VcInd v_trial, v_check;
  ColInd c_trial, c_check, cd_trial, cd_check;
  TraceInd t_trial, t_check;
  XInd xi;
};

// device scalar slots (doubles), mirrored to pinned host memory
enum Slot : int {
  S_GRAD = 0,    // fused operator: C.UU^T part, p.r, r.r, magnitude, epilogue sums [4..7]
  S_PRE = 8,     // pre-pass: |U|_F^2, |colsum|^2
  S_DIFF = 16,   // value change: dT0, p.dT, dT(2rX+dT), trace dT, [4..7] prox sums;
                 // [8..9] colsum-difference pass
  S_VEC = 32,    // streaming kernels
  S_VEC2 = 48,   // streaming kernels (second set)
  S_LAN = 64,    // Lanczos
  S_SCALE = 80,  // |z|^2 and host->device scalar staging
  S_COUNT = 96
};

}  // namespace hallar

// the opaque handle of hallar.h
struct hallar_ctx {
  hallar::Problem P;
  hallar_options opt;
  int device = 0;
  int num_sms = 148;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  hallar::RedBuf red;
  double* d_scal = nullptr;     // [S_COUNT]
  double* h_scal = nullptr;     // pinned mirror
  double* d_colsum = nullptr;   // [4 * kColsumMax]
  std::string last_error;
  int64_t launches = 0;
  // every device buffer the handle owns
  std::vector<void*> owned;
  // staging buffers of the operator entry points (grown on demand)
  void* stage_u = nullptr; size_t stage_u_bytes = 0;
  void* stage_w = nullptr; size_t stage_w_bytes = 0;
  void* stage_wout = nullptr; size_t stage_wout_bytes = 0;
  double* stage_m0 = nullptr; size_t stage_m0_bytes = 0;
  double* stage_m1 = nullptr; size_t stage_m1_bytes = 0;
  double* stage_p0 = nullptr; size_t stage_p0_bytes = 0;
  void* stage_pk = nullptr; size_t stage_pk_bytes = 0;
  void* stage_T = nullptr; size_t stage_T_bytes = 0;     // constraint values in the factor type
  void* stage_y = nullptr; size_t stage_y_bytes = 0;     // second factor (value change, trim)
  double* stage_vc = nullptr; size_t stage_vc_bytes = 0; // r_Y of hallar_value_change
  void* stage_x = nullptr; size_t stage_x_bytes = 0;     // sign vectors (rounding)
  void* stage_pairs = nullptr; size_t stage_pairs_bytes = 0;  // index pairs, entries
  void* eig_stage = nullptr; size_t eig_stage_bytes = 0;
  void* gram_part = nullptr; size_t gram_part_bytes = 0;
  void* trim_gram = nullptr; size_t trim_gram_bytes = 0;
  // Lanczos workspace (basis, vectors, partial rows)
  void* lan_Q = nullptr; size_t lan_Q_bytes = 0;
  void* lan_w = nullptr; size_t lan_w_bytes = 0;
  void* lan_part = nullptr; size_t lan_part_bytes = 0;
  void* lan_h = nullptr; size_t lan_h_bytes = 0;
  // kernel timing (hallar_profile): event pairs pending per kernel class
  bool prof_on = false;
  bool capturing = false;             // kernels are being captured into a graph
  int prof_every = 1;                 // time every prof_every-th launch of a class
  int64_t prof_seen[3] = {0, 0, 0};   // launches of each class since the last clear
  double prof_ms[3] = {0.0, 0.0, 0.0};
  double prof_bytes[3] = {0.0, 0.0, 0.0};  // algorithmic bytes of the timed launches
  double prof_bytes_pad[3] = {0.0, 0.0, 0.0};  // the same with padded factor rows
  int64_t prof_n[3] = {0, 0, 0};
  std::vector<cudaEvent_t> prof_pool;
  std::vector<int> prof_pending;  // (class, start event index), stop = start + 1
  // buffers of the last solve (freed by the next solve or by destroy)
  std::vector<void*> solve_bufs;
  void* sol_U = nullptr; int sol_rank = 0; int sol_ld = 0;
  double* sol_p = nullptr;
};

namespace hallar {
using Ctx = ::hallar_ctx;

// error helpers -------------------------------------------------------------
struct Err {
  hallar_status st;
  std::string msg;
};

#define HL_CUDA(call)                                                             \
  do {                                                                            \
    cudaError_t e__ = (call);                                                     \
    if (e__ != cudaSuccess)                                                       \
      throw ::hallar::Err{e__ == cudaErrorMemoryAllocation ? HALLAR_ENOMEM          \
                                                           : HALLAR_ECUDA,        \
                          std::string(#call) + ": " + cudaGetErrorString(e__)};   \
  } while (0)

#define HL_CHECK_LAUNCH(ctx)                                                      \
  do {                                                                            \
    (ctx)->launches++;                                                            \
    cudaError_t e__ = cudaGetLastError();                                         \
    if (e__ != cudaSuccess)                                                       \
      throw ::hallar::Err{HALLAR_ECUDA, std::string("kernel launch: ") +          \
                                           cudaGetErrorString(e__)};              \
  } while (0)

inline void fail(hallar_status st, const std::string& m) { throw Err{st, m}; }

// buffers -------------------------------------------------------------------
// Device buffers are stream-ordered allocations on the handle's stream
// (cudaMallocAsync / cudaFreeAsync): unlike cudaFree, releasing them does not
// synchronise the device, so handles on different streams -- the serving
// engine's concurrent solves -- never wait for one another's work.
template <class T>
T* dalloc(Ctx* c, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  HL_CUDA(cudaMallocAsync(&p, count * sizeof(T), c->stream));
  c->owned.push_back(p);
  return static_cast<T*>(p);
}
// pinned blocks for the scalar read-backs (S_COUNT doubles) and the host
// mirror of a solve's LoopCtl, recycled across handles (cudaFreeHost would
// synchronise the device)
constexpr int kPinDoubles = S_COUNT + 256;
static_assert(sizeof(LoopCtl) <= 256 * sizeof(double), "LoopCtl outgrew its pinned mirror");
double* pinned_scalars_acquire();
void pinned_scalars_release(double* p);
void dfree(Ctx* c, void* p);
// grow *buf to at least `bytes` (contents not kept)
void* ensure_buffer(Ctx* c, void** buf, size_t* cur_bytes, size_t bytes);
void sync(Ctx* c);
// kernel timing: prof_begin records a start event and returns its token (or
// -1 when timing is off); prof_end records the stop event of that token
int prof_begin(Ctx* c, int cls, OpBytes bytes);
void prof_end(Ctx* c, int token);
void prof_resolve(Ctx* c);  // after a stream sync: add finished pairs
void fetch_scalars(Ctx* c, int first, int count);  // d_scal -> h_scal, then sync

// element size of a factor array for this handle
inline size_t elem_size(const Ctx* c) {
  return c->opt.precision == HALLAR_MIXED ? sizeof(float) : sizeof(double);
}
// leading dimension used internally: r rounded up to 16 bytes
inline int padded_ld(const Ctx* c, int r) {
  int v = c->opt.precision == HALLAR_MIXED ? 4 : 2;
  return (r + v - 1) / v * v;
}

// ---------------------------------------------------------------------------
// kernel launchers (kernels_ops.cu / kernels_vec.cu / lanczos.cu)
// ---------------------------------------------------------------------------
struct GradOut {
  void* W = nullptr;        // [n x ld] or null
  void* resid = nullptr;    // [m] of the factor type, or null (owned constraints;
                            // the trace row is written by the caller)
  double* T = nullptr;      // [m+1] or null (T[0] and the trace row by the caller)
};

OpBytes op_bytes(const Ctx* c, int r, int ld, int factor_arrays, bool writes_resid, bool reads_p,
                 bool reads_rx);
// pre-pass: colsum of U into colsum_out, S_PRE[0] = |U|_F^2, S_PRE[1] = |colsum|^2,
// and C_J * colsum in the factor type at cj_row (kColsumMax entries) when C_J != 0
void launch_colsum(Ctx* c, const void* U, int ld, double* colsum_out, int slot);
// where launch_colsum leaves C_J * colsum in the factor type
inline void* cj_row(const Ctx* c) { return c->d_colsum + 3 * kColsumMax; }
// fused A~(UU^T), shift and SpMM.  Reductions into S_GRAD:
//   [0] C.UU^T without the C_J part, [1] sum p_l r_l, [2] sum r_l^2 (the
//   trace row excluded), [3] sum |p'_l| |A_l.UU^T| + |sparse and diagonal
//   C terms| (the scale of the rounding of g).
// p has the factor's element type (float copy in the mixed form)
void launch_grad(Ctx* c, const void* U, int ld, int r, const void* p, double beta,
                 GradOut out);
// the fused operator with the ADAP-FISTA (EPI_FISTA_Z: S_GRAD[4] = |z|^2) or
// ADAP-AIPP (EPI_AIPP: S_GRAD[4..7] = <V, D>, |D|^2,
// |V - D|^2, <W, y>) epilogue, its arguments read from device memory
void launch_grad_epi(Ctx* c, int epi, int ld, int r, const void* p, const GradInd* gind);
// g(Y) - g(X) pieces into S_DIFF: [0] dT0 (no C_J part) [1] p.dT [2] dT(2rX+dT)
// [3] trace dT = sum <D_i, Y_i + X_i>; rY (if non-null) = rX + dT.
void launch_value_change(Ctx* c, const void* X, const void* Y, int ld, int r,
                         const void* p, const void* rX, void* rY);
// the same with arguments from device memory; y_from_z: Y = cs Z (cs from
// S_GRAD[4] = |Z|^2 and tau), Y stored, and S_DIFF[4..7] = |Y - X|^2,
// <Y - X, (Y + X)/2 - centre>, |Y - centre|^2, <X - Z, Y - X>
void launch_value_change_ind(Ctx* c, bool y_from_z, int ld, int r, const void* p,
                             const VcInd* vind);
// colsum of D = Y - X and of Y + X (for the C_J part of a value change);
// S_DIFF[8] = sum <D_i, Y_i + X_i>, S_DIFF[9] = <colsum D, colsum (Y + X)>
void launch_colsum_diff(Ctx* c, const void* X, const void* Y, int ld, double* sD,
                        double* sS);
// the column-sum pre-passes with arguments from device memory
void launch_colsum_ind(Ctx* c, int ld, const ColInd* cind);
void launch_colsum_diff_ind(Ctx* c, int ld, const ColInd* cind);

// r = 1 operator pieces in FP64 (Frank-Wolfe); resid = A(YY^T) - b (double)
void launch_fw_denom(Ctx* c, const double* y, const double* resid, double tau2, int slot);
// r64 = A(YY^T) - b in double from the stored factor (trace row excluded);
// S[slot] = sum r64^2, S[slot+1] = |Y|_F^2
void launch_resid64(Ctx* c, const void* U, int ld, int r, double* r64, int slot);

// streaming kernels (kernels_vec.cu); reductions into the given slot
void launch_pad_copy(Ctx* c, const void* src, int ld_src, void* dst, int ld_dst, int r_copy,
                     double scale_src);
void launch_scale(Ctx* c, void* U, int ld, double s);
void launch_norm2(Ctx* c, const void* U, int ld, int slot);
void launch_fw_append(Ctx* c, const void* Y, int ld, int r, const double* y, double sY,
                      double sy, void* Ynew, int ld_new, int append);
// m-length FP64 vectors: op 0: a = b + s cc; op 1: slot = <b, cc>; op 2: slot = |b|^2
void launch_dvec(Ctx* c, int op, int64_t len, double* a, const double* b, const double* cc,
                 double s, int slot);
// conversions between double vectors and factor-typed vectors
void launch_to_factor_type(Ctx* c, int64_t len, void* out, const double* in);
void launch_to_double(Ctx* c, int64_t len, double* out, const void* in);
// Gram U^T U (r x r, FP64 result) and out = U Q (Q row-major r x k); the
// mixed form's float Gram runs on the tensor cores (gram_tc.cu)
void launch_gram_tc(Ctx* c, const void* U, int ld, int r, double* G);
void launch_gram(Ctx* c, const void* U, int ld, int r, double* G);
void launch_right_mult(Ctx* c, const void* U, int ld, int r, const double* Q, int k, void* out,
                       int ld_out);

// Lanczos (lanczos.cu)
struct LanczosOut {
  double lambda;
  double resid;
  int iters;
  bool converged;
  int sweeps;  // reorthogonalisation sweeps against the whole basis
};
LanczosOut lanczos_min_eig(Ctx* c, const double* pshift, const double* v0, double tol, int kmax,
                           int max_restarts, double* v_out);
void launch_splitmix(Ctx* c, uint64_t seed, double* out, double mix_scale, const double* base);

// trace-row entry of a residual vector (factor type) from a device scalar:
// r[m-1] = (src ? src[m-1] : 0) + *dscal + add
void launch_trace_fix(Ctx* c, void* r, const void* src, const double* dscal, double add);

// device-side ADAP-AIPP / ADAP-FISTA control (loop.cu)
void launch_loop_reset(Ctx* c, LoopCtl* L);        // attempts = 0 (top of a graph launch)
void launch_aipp_begin(Ctx* c, LoopCtl* L);        // start an ADAP-FISTA call
void launch_fista_ctl(Ctx* c, LoopCtl* L);         // ADAP-FISTA steps 2-5 after a trial
void launch_aipp_ctl(Ctx* c, LoopCtl* L);          // ADAP-AIPP steps 2-3 after a call
void launch_loop_x(Ctx* c, int ld, LoopCtl* L);    // x / x~ updates (XInd of L)
void launch_trace_fix_ind(Ctx* c, const TraceInd* ti, double add);  // dst[m-1] = S_PRE[0] + add

// consumers of a solved factor (consumers.cu): x = sign(U g) (int8, +1 at
// 0); S[slot] = x^T C x without the C_J part, S[slot+1] = sum x; X_ab at pairs
void launch_round_sign(Ctx* c, const void* U, int ld, int r, const double* g, int8_t* x);
void launch_cut(Ctx* c, const int8_t* x, int slot);
void launch_entries(Ctx* c, const void* U, int ld, int r, const int32_t* a, const int32_t* b,
                    int64_t count, double* out);

// solver (solver.cu)
hallar_status solve(Ctx* c, const void* U0, int r0, const double* p0, hallar_result* res);
// rank trim: out (n x ld_out) = Y Q_k, Q_k the k leading eigenvectors of
// Y^T Y; eigs (host, may be null) gets the r Gram eigenvalues, descending
void trim_factor(Ctx* c, const void* Y, int ld, int r, int k, void* out, int ld_out,
                 double* eigs);

// ---------------------------------------------------------------------------
// grid sizing: a fixed grid per (work, items per block) so that reductions
// are deterministic; at most 8 resident 256-thread blocks per SM.
// ---------------------------------------------------------------------------
// blocks of `block` threads of kernel `fn` that one SM holds at once, from
// the occupancy calculator (cached per kernel; at least 1)
int resident_blocks(const void* fn, int block, size_t smem);

// grid of a grid-stride kernel: at most one full wave of resident blocks.
// A grid of a few partial waves leaves SMs idle in the last one; one wave
// of resident blocks keeps every SM busy until the rows run out.
template <class F>
inline int wave_grid(const Ctx* c, F* fn, int64_t work_items, int items_per_block, int block,
                     size_t smem = 0) {
  int64_t g = (work_items + items_per_block - 1) / items_per_block;
  int64_t cap = (int64_t)c->num_sms * resident_blocks((const void*)fn, block, smem);
  if (cap > kMaxBlocks) cap = kMaxBlocks;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

inline int grid_for(const Ctx* c, int64_t work_items, int items_per_block) {
  int64_t g = (work_items + items_per_block - 1) / items_per_block;
  int64_t cap = (int64_t)c->num_sms * 8;
  if (cap > kMaxBlocks) cap = kMaxBlocks;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace hallar
