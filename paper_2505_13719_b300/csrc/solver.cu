// HALLaR driver (Alg. 1) with ADAP-AIPP / ADAP-FISTA (Appendix A) on device
// data.  Every vector (U, the ADAP-FISTA sequences, multipliers, residuals,
// Lanczos vectors) stays in HBM for the whole solve (Section 3.1).  Each
// ADAP-AIPP call runs on the device (loop.cu): its scalar recurrences live in
// a LoopCtl in device memory, and the call is one CUDA graph of two nested
// WHILE nodes (ADAP-FISTA calls, and each call's trials), replayed until the
// call is done, so the host synchronises once per graph launch instead of
// once per trial.  With kernel timing on (hallar_profile) the same kernels
// run one launch at a time, the host reading the loop conditions.  The HLR
// loop, Lanczos, Frank-Wolfe and the AL outer loop stay on the host.
//
// The control flow and its readings of the paper's open points are the same
// as the oracle's:
//   * epsilon_t = max(tol/2 (1 + |pval|), eps_1 eps_decay^(t-1)),
//     eps_1 = eps1_rel (1 + tau^2 ||C||_1); ADAP-AIPP gets rho = epsilon_t / tau;
//   * beta doubles (<= beta_max (1 + ||C||_1)) when ||r_t|| > ||r_{t-1}|| / 4
//     while the relative primal infeasibility is above tol;
//   * ADAP-AIPP: M_j = max(1, Mbar_{j-1}/2), lambda carried across calls
//     (options.lambda_kappa > 0: each call starts at lambda_kappa / beta_t);
//   * ADAP-FISTA: linearisation test with g(y) - g(x~) formed as a
//     difference; V = grad psi(y) - grad psi(x~) + L (x~ - y);
//   * floating point: the step-2 tests of ADAP-FISTA and ADAP-AIPP accept a
//     violation up to 16 u lam sum|terms of g| (u the unit roundoff of the
//     stored factor), and ADAP-AIPP stops when a prox step leaves W
//     unchanged; neither is in the paper, and in FP64 both are inert in
//     practice;
//   * Lanczos start: the previous eigenvector plus 0.1/sqrt(n) times a
//     SplitMix64 vector, Ritz residual <= lanczos_tol_rel epsilon_t / tau^2;
//   * theta = 0: no zero column is appended; rank above r_cap: keep the
//     r_cap leading directions of YY^T (Gram eigenvectors);
//   * termination: eq. termination2, ||C||_1 the induced norm.
// Not in the oracle: a mixed solve whose float factor stalls goes on in FP64
// (options.promote).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

namespace {

// symmetric r x r eigendecomposition by cyclic Jacobi rotations (rank trim)
void jacobi_eig(std::vector<double>& A, int r, std::vector<double>& V, std::vector<double>& w) {
  V.assign((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i) V[(size_t)i * r + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) {
        const double x = A[(size_t)i * r + j];
        tot += x * x;
        if (i != j) off += x * x;
      }
    if (off == 0.0 || off <= 1e-30 * tot) break;
    for (int p = 0; p < r; ++p)
      for (int q = p + 1; q < r; ++q) {
        const double apq = A[(size_t)p * r + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * r + p], aqq = A[(size_t)q * r + q];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < r; ++k) {
          const double akp = A[(size_t)k * r + p], akq = A[(size_t)k * r + q];
          A[(size_t)k * r + p] = cs * akp - sn * akq;
          A[(size_t)k * r + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < r; ++k) {
          const double apk = A[(size_t)p * r + k], aqk = A[(size_t)q * r + k];
          A[(size_t)p * r + k] = cs * apk - sn * aqk;
          A[(size_t)q * r + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < r; ++k) {
          const double vkp = V[(size_t)k * r + p], vkq = V[(size_t)k * r + q];
          V[(size_t)k * r + p] = cs * vkp - sn * vkq;
          V[(size_t)k * r + q] = sn * vkp + cs * vkq;
        }
      }
  }
  w.resize(r);
  for (int i = 0; i < r; ++i) w[i] = A[(size_t)i * r + i];
}

struct GradScal {
  double T0 = 0, pr = 0, rr = 0, nrm2 = 0, g = 0, mag = 0;
};

// ADAP-FISTA calls per graph launch of an ADAP-AIPP call: the host checks
// the time limit between launches
constexpr int kAttemptsPerLaunch = 64;

// a CUDA graph of one ADAP-AIPP call for a factor width
struct LoopGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int ld = -1;
  unsigned long long h_fista = 0, h_aipp = 0;
  int64_t k_top = 0, k_outer = 0, k_trial = 0;  // kernels per launch / call / trial
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    ld = -1;
  }
};

struct Solver {
  Ctx* c;
  Problem& P;
  const hallar_options& o;
  int64_t n = 0, m = 0;
  int ld_max = 0;
  size_t fbytes = 0;  // bytes of one factor buffer
  // factor buffers: pool[3] rotate as the prox centre / y / trial y (the HLR
  // factor Y is pool[ic]); x, x~ and z of ADAP-FISTA
  void* pool[3] = {nullptr, nullptr, nullptr};
  void *xb = nullptr, *xtb = nullptr, *zb = nullptr;
  int ic = 0;  // pool index of the HLR factor
  // p: the multipliers (double, the dual update's precision); pk: the copy of
  // the factor type that the operator kernels read (p itself in FP64);
  // residual vectors have the factor type: rpool[ir] holds A(YY^T) - b at Y
  double *p = nullptr, *pshift = nullptr;
  double* r64 = nullptr;  // A(YY^T) - b in double at the HLR factor
  void* pk = nullptr;
  void* rpool[2] = {nullptr, nullptr};
  void* rX = nullptr;
  int ir = 0;
  double *v = nullptr, *vprev = nullptr, *v0 = nullptr;
  LoopCtl* d_ctl = nullptr;  // device
  LoopCtl* h_ctl = nullptr;  // pinned host mirror
  LoopGraph graph;
  int rank = 0, ld = 0;
  double beta = 1.0, lam = 1.0, Mbar = 1.0, p_tr = 0.0, b_tr = 0.0;
  int prec0 = HALLAR_FP64;  // the handle's form (a promoted solve returns to it)
  int stalls_t = 0;         // ADAP-AIPP calls of this AL iteration that stalled
  hallar_result R{};
  std::chrono::steady_clock::time_point t0;

  explicit Solver(Ctx* cc) : c(cc), P(cc->P), o(cc->opt), prec0(cc->opt.precision) {}
  ~Solver() { graph.release(); }

  void* Y() const { return pool[ic]; }
  double tau() const { return std::sqrt(P.tau2); }
  // unit roundoff of the stored factor: rounding the iterates moves g by up
  // to about u * mag; the acceptance tests of ADAP-FISTA step 2 and
  // ADAP-AIPP step 2 allow kRoundSlack times that
  double unit() const { return o.precision == HALLAR_MIXED ? 0x1p-24 : 0x1p-53; }
  static constexpr double kRoundSlack = 16.0;
  bool needs_colsum() const { return P.C_J != 0.0 || P.has_trace; }
  // the solver's own buffers (kept after the solve for hallar_get_solution)
  std::vector<void*> mine;
  template <class T>
  T* salloc(size_t count) {
    T* q = dalloc<T>(c, count);
    mine.push_back(q);
    return q;
  }
  void* fbuf() { return salloc<unsigned char>(fbytes); }

  void setup() {
    n = P.n;
    m = P.m;
    ld_max = padded_ld(c, o.r_cap + 1);
    fbytes = (size_t)n * ld_max * elem_size(c);
    for (auto& b : pool) b = fbuf();
    xb = fbuf();
    xtb = fbuf();
    zb = fbuf();
    p = salloc<double>(m);
    pk = o.precision == HALLAR_MIXED ? (void*)salloc<float>(m) : (void*)p;
    for (auto& b : rpool) b = salloc<unsigned char>(m * elem_size(c));
    rX = salloc<unsigned char>(m * elem_size(c));
    pshift = salloc<double>(m);
    r64 = salloc<double>(m);
    v = salloc<double>(n);
    vprev = salloc<double>(n);
    v0 = salloc<double>(n);
    d_ctl = salloc<LoopCtl>(1);
    h_ctl = reinterpret_cast<LoopCtl*>(c->h_scal + S_COUNT);
    if (P.has_trace) {
      HL_CUDA(cudaMemcpyAsync(&b_tr, P.b + (m - 1), sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
      HL_CUDA(cudaStreamSynchronize(c->stream));
    }
  }

  // the kernels' copy of p after p changed
  void refresh_pk() {
    if (pk != (void*)p) launch_to_factor_type(c, m, pk, p);
  }

  // enqueue: pre-pass + fused operator at U (W and resid optional)
  void grad_enqueue(const void* U, void* W, void* resid) {
    if (needs_colsum()) launch_colsum(c, U, ld, c->d_colsum, S_PRE);
    launch_grad(c, U, ld, rank, pk, beta, GradOut{W, resid, nullptr});
    if (resid && P.has_trace) launch_trace_fix(c, resid, nullptr, c->d_scal + S_PRE, -b_tr);
    R.grad_evals++;
  }
  GradScal grad_read() const {
    const double* h = c->h_scal;
    GradScal s;
    s.nrm2 = h[S_PRE];
    s.T0 = h[S_GRAD] + P.C_J * h[S_PRE + 1];
    s.pr = h[S_GRAD + 1];
    s.rr = h[S_GRAD + 2];
    s.mag = h[S_GRAD + 3] + std::fabs(P.C_J) * h[S_PRE + 1];
    if (P.has_trace) {
      const double rt = s.nrm2 - b_tr;
      s.pr += p_tr * rt;
      s.rr += rt * rt;
      s.mag += std::fabs(p_tr + beta * rt) * s.nrm2;
    }
    s.g = s.T0 + s.pr + 0.5 * beta * s.rr;
    return s;
  }
  void fetch() { fetch_scalars(c, 0, S_COUNT); }

  void check_time() {
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > o.time_limit_s) throw Err{HALLAR_ETIMEOUT, "time limit reached"};
  }

  // ---- the device-side ADAP-AIPP loop -------------------------------------
  // one ADAP-FISTA trial: operator at x~ with the z epilogue, the value
  // change to y = P_B(z) with the prox sums, control, x / x~ updates
  void enqueue_trial() {
    if (needs_colsum()) launch_colsum_ind(c, ld, &d_ctl->c_trial);
    launch_grad_epi(c, EPI_FISTA_Z, ld, rank, pk, &d_ctl->g_trial);
    if (P.C_J != 0.0) launch_colsum_diff_ind(c, ld, &d_ctl->cd_trial);
    launch_value_change_ind(c, true, ld, rank, pk, &d_ctl->v_trial);
    launch_fista_ctl(c, d_ctl);
    launch_loop_x(c, ld, d_ctl);
  }
  // after an ADAP-FISTA call: ADAP-AIPP step 2 at its output y
  void enqueue_check() {
    if (needs_colsum()) launch_colsum_ind(c, ld, &d_ctl->c_check);
    launch_grad_epi(c, EPI_AIPP, ld, rank, pk, &d_ctl->g_check);
    if (P.has_trace) launch_trace_fix_ind(c, &d_ctl->t_check, -b_tr);
    if (P.C_J != 0.0) launch_colsum_diff_ind(c, ld, &d_ctl->cd_check);
    launch_value_change_ind(c, false, ld, rank, pk, &d_ctl->v_check);
    launch_aipp_ctl(c, d_ctl);
  }

  // Capture the ADAP-AIPP call as a graph: [reset] -> WHILE(aipp) {
  // begin -> WHILE(fista) { trial } -> check }.  Nothing allocates while
  // capturing (every buffer exists), and kernel timing is off.
  void build_graph() {
    graph.release();
    cudaStream_t s = c->stream;
    const int64_t launches0 = c->launches;
    c->capturing = true;
    struct CaptureGuard {
      Ctx* c;
      ~CaptureGuard() {
        c->capturing = false;
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(c->stream, &st) == cudaSuccess &&
            st != cudaStreamCaptureStatusNone) {
          cudaGraph_t junk = nullptr;
          cudaStreamEndCapture(c->stream, &junk);
          if (junk) cudaGraphDestroy(junk);
        }
        cudaGetLastError();
      }
    } guard{c};
    HL_CUDA(cudaGraphCreate(&graph.graph, 0));
    cudaGraphConditionalHandle ha, hf;
    HL_CUDA(cudaGraphConditionalHandleCreate(&ha, graph.graph, 1, cudaGraphCondAssignDefault));
    // top level: reset, then the ADAP-AIPP WHILE node
    HL_CUDA(cudaStreamBeginCaptureToGraph(s, graph.graph, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    launch_loop_reset(c, d_ctl);
    cudaGraph_t body_a = add_while(s, ha);
    HL_CUDA(cudaStreamEndCapture(s, &graph.graph));
    graph.k_top = c->launches - launches0;
    // ADAP-AIPP body: begin, the ADAP-FISTA WHILE node, the step-2 check
    HL_CUDA(cudaGraphConditionalHandleCreate(&hf, body_a, 0, 0));
    int64_t l1 = c->launches;
    HL_CUDA(cudaStreamBeginCaptureToGraph(s, body_a, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    launch_aipp_begin(c, d_ctl);
    cudaGraph_t body_f = add_while(s, hf);
    enqueue_check();
    cudaGraph_t tmp = body_a;
    HL_CUDA(cudaStreamEndCapture(s, &tmp));
    graph.k_outer = c->launches - l1;
    // ADAP-FISTA body: one trial
    l1 = c->launches;
    HL_CUDA(cudaStreamBeginCaptureToGraph(s, body_f, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    enqueue_trial();
    tmp = body_f;
    HL_CUDA(cudaStreamEndCapture(s, &tmp));
    graph.k_trial = c->launches - l1;
    c->launches = launches0;  // captured, not launched
    HL_CUDA(cudaGraphInstantiate(&graph.exec, graph.graph, 0));
    graph.ld = ld;
    graph.h_fista = (unsigned long long)hf;
    graph.h_aipp = (unsigned long long)ha;
  }

  // add a WHILE node after the capture's current dependencies; the capture
  // continues after it.  Returns the node's body graph.
  cudaGraph_t add_while(cudaStream_t s, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    HL_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &ndeps));
    if (st != cudaStreamCaptureStatusActive) fail(HALLAR_ECUDA, "graph capture is not active");
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    HL_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
    HL_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                cudaStreamSetCaptureDependencies));
    return np.conditional.phGraph_out[0];
  }

  // ADAP-AIPP (Appendix A) from Y = pool[ic]; on return pool[ic] holds W,
  // rpool[ir] its residuals, *gs the operator scalars at W and *GdotX
  // G . WW^T = <(C + A*(p'))W, W>.
  void aipp(double rho, GradScal* gs, double* GdotX) {
    // residuals at the centre and |centre|^2 (trace row)
    grad_enqueue(Y(), nullptr, rpool[ir]);
    fetch();
    const double nrm_ctr2 = c->h_scal[S_PRE];
    if (o.lambda_kappa > 0.0) lam = o.lambda_kappa / beta;  // a fresh start per call
    const bool eager = c->prof_on;  // per-kernel timing needs launches of their own
    LoopCtl& H = *h_ctl;
    std::memset(&H, 0, sizeof(LoopCtl));
    for (int k = 0; k < 3; ++k) H.pool[k] = pool[k];
    H.xb = xb;
    H.xtb = xtb;
    H.zb = zb;
    H.rpool[0] = rpool[0];
    H.rpool[1] = rpool[1];
    H.rX = rX;
    H.i_ctr = ic;
    H.i_rctr = ir;
    H.mixed = o.precision == HALLAR_MIXED;
    H.has_trace = P.has_trace;
    H.beta = beta;
    H.tau = tau();
    H.chi = o.chi;
    H.sigma = o.sigma;
    H.mu = 0.5;
    H.slack_u = kRoundSlack * unit();
    H.rho = rho;
    H.C_J = P.C_J;
    H.b_tr = b_tr;
    H.p_tr = p_tr;
    H.max_fista = o.max_fista;
    H.max_aipp = o.max_aipp;
    H.attempt_cap = eager ? (1 << 30) : kAttemptsPerLaunch;
    H.trial_cap = o.max_fista * 128;
    H.lam = lam;
    H.Mbar = Mbar;
    H.nrm_ctr2 = nrm_ctr2;
    H.graph_mode = eager ? 0 : 1;
    H.verbose = o.verbose;
    if (!eager) {
      if (graph.ld != ld) build_graph();
      H.h_fista = graph.h_fista;
      H.h_aipp = graph.h_aipp;
    }
    HL_CUDA(cudaMemcpyAsync(d_ctl, &H, sizeof(LoopCtl), cudaMemcpyHostToDevice, c->stream));
    if (eager) {
      int32_t* flag = reinterpret_cast<int32_t*>(c->h_scal + S_SCALE + 6);
      for (;;) {
        launch_aipp_begin(c, d_ctl);
        do {
          enqueue_trial();
          HL_CUDA(cudaMemcpyAsync(flag, &d_ctl->cont_fista, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, c->stream));
          sync(c);
        } while (*flag);
        enqueue_check();
        HL_CUDA(cudaMemcpyAsync(flag, &d_ctl->cont_aipp, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        if (!*flag) break;
        check_time();
      }
      HL_CUDA(cudaMemcpyAsync(&H, d_ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, c->stream));
      sync(c);
    } else {
      for (;;) {
        HL_CUDA(cudaGraphLaunch(graph.exec, c->stream));
        HL_CUDA(cudaMemcpyAsync(&H, d_ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        c->launches += graph.k_top;
        if (H.done || H.error) break;
        check_time();
      }
      c->launches += graph.k_outer * H.n_attempts + graph.k_trial * H.n_trials;
    }
    if (H.stall_exit) stalls_t++;
    R.fista_iters += (int32_t)H.n_fista_iters;
    R.fista_failures += (int32_t)H.n_fista_fail;
    R.aipp_iters += (int32_t)H.n_aipp_iters;
    R.grad_evals += H.n_grads;
    R.value_evals += H.n_values;
    if (H.error == HALLAR_ENUMERIC)
      throw Err{HALLAR_ENUMERIC, "non-finite ADAP-FISTA step or prox stepsize underflow"};
    if (H.error) throw Err{(hallar_status)H.error, "ADAP-FISTA trial limit reached"};
    lam = H.lam;
    Mbar = H.Mbar;
    ic = H.i_ctr;
    ir = H.i_rctr;
    gs->T0 = H.gT0;
    gs->pr = H.gpr;
    gs->rr = H.grr;
    gs->nrm2 = H.gnrm2;
    gs->mag = H.gmag;
    gs->g = H.gT0 + H.gpr + 0.5 * beta * H.grr;
    *GdotX = H.gWU;
    if (o.verbose >= 2)
      std::fprintf(stderr, "[aipp] lam=%.3e Mbar=%.3e |R|=%.3e rho=%.3e fista=%lld trials=%lld\n",
                   lam, Mbar, H.Rn, rho, H.n_fista_iters, H.n_trials);
  }

  // r64 = A(YY^T) - b at the HLR factor, every product in double from the
  // stored factor (the trace row from |Y|_F^2); gs->rr and gs->nrm2 are
  // replaced by the double values.  The dual update, the Lanczos shift, the
  // Frank-Wolfe step and the KKT residual read these (in the mixed form the
  // operator kernels' float residuals would carry rounding that beta
  // amplifies into the multipliers).
  void resid64(GradScal* gs) {
    launch_resid64(c, Y(), ld, rank, r64, S_VEC2 + 10);
    fetch();
    double rr = c->h_scal[S_VEC2 + 10];
    const double nrm2 = c->h_scal[S_VEC2 + 11];
    if (P.has_trace) {
      const double rt = nrm2 - b_tr;
      rr += rt * rt;
      c->h_scal[S_SCALE + 5] = rt;
      HL_CUDA(cudaMemcpyAsync(r64 + (m - 1), c->h_scal + S_SCALE + 5, sizeof(double),
                              cudaMemcpyHostToDevice, c->stream));
    }
    gs->rr = rr;
    gs->nrm2 = nrm2;
  }

  // the pool index other than ic and `busy` (the destination of a new factor)
  int free_slot() const { return (ic + 1) % 3; }

  void trim_rank() {
    // keep the r_cap leading eigenvectors of Y^T Y (Y = pool[ic], rank columns)
    const int k = o.r_cap;
    const int ld_new = padded_ld(c, k);
    const int dst = free_slot();
    trim_factor(c, Y(), ld, rank, k, pool[dst], ld_new, nullptr);
    ic = dst;
    rank = k;
    ld = ld_new;
    R.trims++;
  }

  // ---- promotion of a mixed solve to FP64 ---------------------------------
  // A float factor resolves each entry to 2^-24 of its size.  Once beta has
  // grown so far that ADAP-AIPP's prox steps round away (W unchanged while
  // |R| > rho), neither ADAP-AIPP nor the Frank-Wolfe update (sqrt(1 - alpha)
  // rounds to 1) can move the iterate, and the residual stops falling.  (A
  // step that leaves W bitwise unchanged also gives V = 0, so such a call
  // reports |R| = 0: the sign is the repeated stall, whatever |R| is.)  The
  // solve then goes on in FP64 from where it is: the factor is widened (exact),
  // p, beta, lambda and Mbar carry over, and every kernel from here on is the
  // FP64 instantiation.  The float ld (a multiple of 4) is a valid FP64 ld.
  static constexpr int kPromoteStalls = 4;

  void release_buf(void*& q) {
    auto it = std::find(mine.begin(), mine.end(), q);
    if (it != mine.end()) mine.erase(it);
    dfree(c, q);
    q = nullptr;
  }

  void promote(int t) {
    const size_t fb64 = (size_t)n * ld_max * sizeof(double);
    double* y64 = salloc<double>((size_t)n * ld_max);
    launch_to_double(c, n * (int64_t)ld, y64, Y());  // before the form changes
    for (auto& b : pool) release_buf(b);
    release_buf(xb);
    release_buf(xtb);
    release_buf(zb);
    for (auto& b : rpool) release_buf(b);
    release_buf(rX);
    if (pk != (void*)p) release_buf(pk);
    c->opt.precision = HALLAR_FP64;  // o is the handle's options: unit(), H.mixed follow
    fbytes = fb64;
    pool[0] = y64;
    pool[1] = fbuf();
    pool[2] = fbuf();
    xb = fbuf();
    xtb = fbuf();
    zb = fbuf();
    for (auto& b : rpool) b = salloc<double>(m);
    rX = salloc<double>(m);
    pk = p;
    ic = 0;
    ir = 0;
    graph.release();  // the captured kernels are the float instantiations
    R.promoted_at = t;
    if (o.verbose)
      std::fprintf(stderr, "[hallar] t=%d mixed form stalled (%d ADAP-AIPP calls): FP64 from here\n",
                   t, stalls_t);
  }

  // after a promoted solve: the handle's form again, and the factor in it
  // for hallar_get_solution
  void narrow_solution() {
    if (!R.promoted_at || o.precision == prec0) {
      c->opt.precision = prec0;
      return;
    }
    void* y32 = salloc<float>((size_t)n * ld);
    const void* y64 = Y();
    c->opt.precision = prec0;
    launch_to_factor_type(c, n * (int64_t)ld, y32, (const double*)y64);
    pool[ic] = y32;
    graph.release();
  }

  hallar_status run(const void* U0d, int r0, const double* p0d, hallar_result* out) {
    t0 = std::chrono::steady_clock::now();
    const double tauv = tau();
    // initial factor: padded copy, projected onto the ball
    rank = r0;
    ld = padded_ld(c, r0);
    ic = 0;
    ir = 0;
    launch_pad_copy(c, U0d, r0, Y(), ld, r0, 1.0);
    launch_norm2(c, Y(), ld, S_VEC);
    if (p0d) HL_CUDA(cudaMemcpyAsync(p, p0d, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    else HL_CUDA(cudaMemsetAsync(p, 0, m * sizeof(double), c->stream));
    refresh_pk();
    fetch();
    const double nU = std::sqrt(c->h_scal[S_VEC]);
    if (nU > tauv) launch_scale(c, Y(), ld, tauv / nU);
    if (P.has_trace) {
      HL_CUDA(cudaMemcpyAsync(&c->h_scal[S_SCALE + 3], p + (m - 1), sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
      sync(c);
      p_tr = c->h_scal[S_SCALE + 3];
    }
    beta = o.beta0;
    lam = o.lambda0;
    Mbar = 1.0;
    const double eps1 = o.eps1_rel * (1.0 + P.tau2 * P.c_norm1);
    const double beta_cap = o.beta_max * (1.0 + P.c_norm1);  // in units of 1 + |C|_1
    double prev_rnorm = INFINITY;
    bool have_vprev = false;
    grad_enqueue(Y(), nullptr, nullptr);  // pval at the start point
    fetch();
    double pval_now = grad_read().T0;
    double theta = 0.0, lam_min = 0.0;
    GradScal gs;
    hallar_status st = HALLAR_ENOTCONV;
    for (int t = 1; t <= o.max_outer; ++t) {
      R.outer_iters++;
      stalls_t = 0;
      const double eps_floor = 0.5 * o.tol * (1.0 + std::fabs(pval_now));
      const double eps_t = std::fmax(eps_floor, eps1 * std::pow(o.eps_decay, t - 1));
      const double rho_t = eps_t / std::fmax(tauv, 1e-300);
      for (int hl = 0; hl < o.max_hlr; ++hl) {                      // HLR
        R.hlr_iters++;
        double GdotX = 0.0;                                         // G . YY^T = <GY, Y>
        aipp(rho_t, &gs, &GdotX);                                   // step 6
        resid64(&gs);                                               // r(Y) in double
        launch_dvec(c, 0, m, pshift, p, r64, beta, -1);             // p' = p + beta r(Y)
        const uint64_t sd = o.seed + 7919ull * (uint64_t)R.hlr_iters;
        launch_splitmix(c, sd, v0, 0.1 / std::sqrt((double)n), have_vprev ? vprev : nullptr);
        const double eig_tol = o.lanczos_tol_rel * eps_t / P.tau2;  // step 7
        const LanczosOut le = lanczos_min_eig(c, pshift, v0, eig_tol, o.lanczos_kmax, 50, v);
        R.lanczos_iters += le.iters;
        HL_CUDA(cudaMemcpyAsync(vprev, v, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        have_vprev = true;
        theta = std::fmax(-le.lambda, 0.0);                         // eq. FW subproblem
        lam_min = le.lambda;
        const double gap = GdotX + P.tau2 * theta;
        if (gap <= eps_t) break;                                    // step 8
        if (hl + 1 == o.max_hlr) break;                             // HLR limit: keep Y
        // Frank-Wolfe step (eqs. FW stepsize, tilde Y)              // step 11
        launch_fw_denom(c, v, r64, theta > 0.0 ? P.tau2 : 0.0, S_VEC2);
        fetch();
        double ssq = c->h_scal[S_VEC2];
        if (P.has_trace) {
          const double dtr = gs.nrm2 - (theta > 0.0 ? P.tau2 * c->h_scal[S_VEC2 + 1] : 0.0);
          ssq += dtr * dtr;
        }
        const double denom = beta * ssq;
        const double alpha = denom <= 0.0 ? 1.0 : std::fmin(gap / denom, 1.0);
        R.fw_steps++;
        int ldn = ld;
        const int dst = free_slot();
        if (theta > 0.0) {
          if (alpha >= 1.0) {
            ldn = padded_ld(c, 1);
            launch_fw_append(c, Y(), ld, 0, v, 0.0, tauv, pool[dst], ldn, 1);
            rank = 1;
          } else {
            ldn = padded_ld(c, rank + 1);
            launch_fw_append(c, Y(), ld, rank, v, std::sqrt(1.0 - alpha),
                             std::sqrt(alpha) * tauv, pool[dst], ldn, 1);
            rank += 1;
          }
        } else if (alpha >= 1.0) {
          ldn = padded_ld(c, 1);
          launch_fw_append(c, Y(), ld, 0, v, 0.0, 0.0, pool[dst], ldn, 0);
          rank = 1;
        } else {
          launch_fw_append(c, Y(), ld, rank, v, std::sqrt(1.0 - alpha), 0.0, pool[dst], ld, 0);
        }
        ld = ldn;
        ic = dst;
        if (rank > o.r_cap) trim_rank();
        check_time();
      }
      // U_t = Y; dual update p_t = p + beta r (step 14), r in double
      launch_dvec(c, 0, m, p, p, r64, beta, -1);
      refresh_pk();
      if (P.has_trace) p_tr += beta * (gs.nrm2 - b_tr);
      launch_dvec(c, 1, m, nullptr, P.b, p, 0.0, S_VEC2 + 4);
      fetch();
      const double btp = c->h_scal[S_VEC2 + 4];
      const double pval = gs.T0;
      const double dval = -btp - P.tau2 * theta;
      const double rnorm = std::sqrt(gs.rr);
      const double rp = rnorm / (1.0 + P.b_norm1);
      const double rg = std::fabs(pval - dval) / (1.0 + std::fabs(pval) + std::fabs(dval));
      const double rd = std::fmax(0.0, -(lam_min + theta)) / (1.0 + P.c_norm1);
      R.pval = pval;
      R.dval = dval;
      R.theta = theta;
      R.lam_min_S = lam_min + theta;
      R.rel_primal = rp;
      R.rel_gap = rg;
      R.rel_dual = rd;
      R.kkt = std::fmax(rp, std::fmax(rg, rd));
      R.beta = beta;
      R.rank = rank;
      if (o.verbose)
        std::fprintf(stderr,
                     "[hallar] t=%d rank=%d beta=%.3g eps=%.3g pval=%.12g dval=%.12g rp=%.2e "
                     "rg=%.2e grads=%lld fista=%d lanczos=%d %.3fs\n",
                     t, rank, beta, eps_t, pval, dval, rp, rg, (long long)R.grad_evals,
                     R.fista_iters, R.lanczos_iters,
                     std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
      if (!std::isfinite(R.kkt)) throw Err{HALLAR_ENUMERIC, "non-finite KKT residual"};
      if (R.kkt <= o.tol) {                                         // step 15
        st = HALLAR_OK;
        R.converged = 1;
        break;
      }
      if (o.promote && o.precision == HALLAR_MIXED && stalls_t >= kPromoteStalls) promote(t);
      // the penalty grows only while primal infeasibility is above the tolerance
      if (rp > o.tol && rnorm > 0.25 * prev_rnorm) beta = std::fmin(2.0 * beta, beta_cap);
      prev_rnorm = rnorm;
      pval_now = pval;
      check_time();
    }
    narrow_solution();
    sync(c);
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    c->sol_U = Y();
    c->sol_rank = rank;
    c->sol_ld = ld;
    c->sol_p = p;
    if (out) *out = R;
    return st;
  }
};

}  // namespace

// Rank trim (not in the paper; the rank cap of hallar_options): out = Y Q_k
// with Q_k the k leading eigenvectors of the Gram Y^T Y (FP64, cyclic
// Jacobi on the host), so out out^T is the best rank-k approximation of
// YY^T (Eckart-Young).  eigs (host, may be null) receives the r Gram
// eigenvalues in descending order.
void trim_factor(Ctx* c, const void* Y, int ld, int r, int k, void* out, int ld_out,
                 double* eigs) {
  double* gram = (double*)ensure_buffer(c, &c->trim_gram, &c->trim_gram_bytes,
                                        (size_t)r * (r > k ? r : k) * sizeof(double));
  launch_gram(c, Y, ld, r, gram);
  std::vector<double> G((size_t)r * r), V, w;
  HL_CUDA(cudaMemcpyAsync(G.data(), gram, G.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  sync(c);
  jacobi_eig(G, r, V, w);
  std::vector<int> idx(r);
  for (int i = 0; i < r; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] > w[b]; });
  if (eigs)
    for (int i = 0; i < r; ++i) eigs[i] = w[idx[i]];
  std::vector<double> Qk((size_t)r * k, 0.0);
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < k && b < r; ++b) Qk[(size_t)a * k + b] = V[(size_t)a * r + idx[b]];
  HL_CUDA(cudaMemcpyAsync(gram, Qk.data(), Qk.size() * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  launch_right_mult(c, Y, ld, r, gram, k, out, ld_out);
  sync(c);
}

hallar_status solve(Ctx* c, const void* U0, int r0, const double* p0, hallar_result* res) {
  // the previous solve's buffers are released before a new solve allocates
  for (void* q : c->solve_bufs) dfree(c, q);
  c->solve_bufs.clear();
  c->sol_U = nullptr;
  c->sol_p = nullptr;
  const int64_t launches0 = c->launches;
  Solver s(c);
  auto keep_buffers = [&]() { c->solve_bufs = s.mine; };
  try {
    s.setup();
    const hallar_status st = s.run(U0, r0, p0, res);
    keep_buffers();
    if (res) res->kernel_launches = c->launches - launches0;
    return st;
  } catch (const Err& e) {
    // a promoted solve leaves the handle in its own form, with a solution in it
    try {
      s.narrow_solution();
    } catch (const Err&) {
      c->opt.precision = s.prec0;
      s.pool[s.ic] = nullptr;
    }
    keep_buffers();
    s.R.seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - s.t0).count();
    if (res) {
      *res = s.R;
      res->kernel_launches = c->launches - launches0;
    }
    if (e.st == HALLAR_ETIMEOUT && s.pool[s.ic]) {
      c->sol_U = s.Y();
      c->sol_rank = s.rank;
      c->sol_ld = s.ld;
      c->sol_p = s.p;
    }
    throw;
  }
}

}  // namespace hallar
