// HALLaR driver (Alg. 1) with ADAP-AIPP / ADAP-FISTA (Appendix A) on device
// data.  The host holds only scalars: every vector (U, the FISTA sequences,
// multipliers, residuals, Lanczos vectors) stays in HBM for the whole solve
// (Section 3.1), and each FISTA iteration costs one device->host transfer of
// the reduction slots.  The control flow and its readings of the paper's
// open points are the same as the oracle's:
//   * epsilon_t = max(tol/2 (1 + |pval|), eps_1 eps_decay^(t-1)),
//     eps_1 = eps1_rel (1 + tau^2 ||C||_1); ADAP-AIPP gets rho = epsilon_t / tau;
//   * beta doubles (<= beta_max) when ||r_t|| > ||r_{t-1}|| / 4 while the
//     relative primal infeasibility is above tol;
//   * ADAP-AIPP: M_j = max(1, Mbar_{j-1}/2), lambda carried across calls;
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
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
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

struct Solver {
  Ctx* c;
  Problem& P;
  const hallar_options& o;
  int64_t n = 0, m = 0;
  int ld_max = 0;
  size_t fbytes = 0;  // bytes of one factor buffer
  void *Ytil = nullptr, *ctr = nullptr, *x = nullptr, *y = nullptr, *xt = nullptr, *z = nullptr;
  void *ynew = nullptr, *Wg = nullptr, *Wy = nullptr, *tmp = nullptr;
  // p: the multipliers (double, the dual update's precision); pk: the copy of
  // the factor type that the operator kernels read (p itself in FP64);
  // residual vectors have the factor type
  double *p = nullptr, *pshift = nullptr;
  void *pk = nullptr, *r_ctr = nullptr, *rX = nullptr, *rY = nullptr;
  double *v = nullptr, *vprev = nullptr, *v0 = nullptr;
  int rank = 0, ld = 0;
  double beta = 1.0, lam = 1.0, Mbar = 1.0, p_tr = 0.0, b_tr = 0.0;
  hallar_result R{};
  std::chrono::steady_clock::time_point t0;

  explicit Solver(Ctx* cc) : c(cc), P(cc->P), o(cc->opt) {}

  double tau() const { return std::sqrt(P.tau2); }
  // unit roundoff of the stored factor: rounding the iterates moves g by up
  // to about u * mag; the acceptance tests of ADAP-FISTA step 2 and
  // ADAP-AIPP step 2 allow kRoundSlack times that
  double unit() const { return o.precision == HALLAR_MIXED ? 0x1p-24 : 0x1p-53; }
  static constexpr double kRoundSlack = 16.0;
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
    Ytil = fbuf(); ctr = fbuf(); x = fbuf(); y = fbuf(); xt = fbuf(); z = fbuf();
    ynew = fbuf(); Wg = fbuf(); Wy = fbuf(); tmp = fbuf();
    p = salloc<double>(m);
    pk = o.precision == HALLAR_MIXED ? (void*)salloc<float>(m) : (void*)p;
    r_ctr = salloc<unsigned char>(m * elem_size(c));
    rX = salloc<unsigned char>(m * elem_size(c));
    rY = salloc<unsigned char>(m * elem_size(c));
    pshift = salloc<double>(m);
    v = salloc<double>(n);
    vprev = salloc<double>(n);
    v0 = salloc<double>(n);
    if (P.has_trace) {
      HL_CUDA(cudaMemcpyAsync(&b_tr, P.b + (m - 1), sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
      HL_CUDA(cudaStreamSynchronize(c->stream));
    }
  }

  void copyf(void* dst, const void* src) {
    HL_CUDA(cudaMemcpyAsync(dst, src, (size_t)n * ld * elem_size(c), cudaMemcpyDeviceToDevice,
                            c->stream));
  }

  // trace-row entry of a residual vector from a device scalar
  void trace_fix(void* r, const void* src, const double* dscal, double add) {
    launch_trace_fix(c, r, src, dscal, add);
  }
  // the kernels' copy of p after p changed
  void refresh_pk() {
    if (pk != (void*)p) launch_to_factor_type(c, m, pk, p);
  }

  // enqueue: pre-pass + fused operator at U (W and resid optional)
  void grad_enqueue(const void* U, void* W, void* resid) {
    if (P.C_J != 0.0 || P.has_trace) launch_colsum(c, U, ld, c->d_colsum, S_PRE);
    launch_grad(c, U, ld, rank, pk, beta, GradOut{W, resid, nullptr});
    if (resid && P.has_trace) trace_fix(resid, nullptr, c->d_scal + S_PRE, -b_tr);
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
  // enqueue: g(Y) - g(X) pieces (rY = A(YY^T) - b when rY != null)
  void change_enqueue(const void* X, const void* Yv, const void* rXv, void* rYv) {
    if (P.C_J != 0.0)
      launch_colsum_diff(c, X, Yv, ld, c->d_colsum + kColsumMax, c->d_colsum + 2 * kColsumMax);
    launch_value_change(c, X, Yv, ld, rank, pk, rXv, rYv);
    if (rYv && P.has_trace) trace_fix(rYv, rXv, c->d_scal + S_DIFF + 3, 0.0);
    R.value_evals++;
  }
  double change_read(double nrmX2) const {
    const double* h = c->h_scal;
    const double dT0 = h[S_DIFF] + (P.C_J != 0.0 ? P.C_J * h[S_DIFF + 5] : 0.0);
    double pd = h[S_DIFF + 1], q = h[S_DIFF + 2];
    if (P.has_trace) {
      const double dt = h[S_DIFF + 3];
      const double rx = nrmX2 - b_tr;
      pd += p_tr * dt;
      q += dt * (2.0 * rx + dt);
    }
    return dT0 + pd + 0.5 * beta * q;
  }
  void fetch() { fetch_scalars(c, 0, S_COUNT); }

  void check_time() {
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > o.time_limit_s) throw Err{HALLAR_ETIMEOUT, "time limit reached"};
  }

  // step 2's a_j for the trial stepsize Ln (the positive root of
  // (Ln - mu) a^2 = tk (A + a))
  static double next_a(double tk, double A, double Ln, double mu) {
    return (tk + std::sqrt(tk * tk + 4.0 * tk * A * (Ln - mu))) / (2.0 * (Ln - mu));
  }

  // ADAP-FISTA on psi_s = lam g + 1/2 |. - ctr|^2 from x0 = ctr.
  // On success ynew holds y, z its unprojected step and *Lout the final L.
  bool fista(double lamv, double mu, double L0, double* Lout) {
    copyf(x, ctr);
    copyf(y, ctr);
    double A = 0.0, tk = 1.0, L = L0;
    const double tauv = tau();
    bool xt_ready = false;  // x~ of the first trial already formed by step 3's pass
    for (int it = 0; it < o.max_fista; ++it) {
      R.fista_iters++;
      if ((it & 15) == 15) check_time();
      double Ln = L, a = 0.0, d2 = 0.0, dy0 = 0.0;
      for (;;) {                                                 // step 2
        a = next_a(tk, A, Ln, mu);
        if (xt_ready) xt_ready = false;
        else if (A == 0.0) copyf(xt, x);
        else launch_fista_xt(c, xt, y, x, A, a, ld);
        grad_enqueue(xt, Wg, rX);
        launch_fista_z(c, z, xt, Wg, ctr, lamv, Ln, ld);
        launch_fista_y(c, ynew, z, xt, ctr, Wg, lamv, tauv, ld);
        change_enqueue(xt, ynew, rX, rY);
        fetch();
        const double nrm_xt2 = c->h_scal[S_PRE];
        d2 = c->h_scal[S_VEC];
        const double gd = c->h_scal[S_VEC + 1];
        const double dlin = c->h_scal[S_VEC + 2];
        dy0 = c->h_scal[S_VEC + 3];
        const double dpsi = lamv * change_read(nrm_xt2) + dlin;
        const double slack = kRoundSlack * unit() * lamv * grad_read().mag;
        if (!std::isfinite(dpsi) || !std::isfinite(gd))
          throw Err{HALLAR_ENUMERIC, "non-finite ADAP-FISTA step"};
        if (o.verbose >= 3)
          std::fprintf(stderr, "[fista] it=%d L=%.3e d2=%.3e gd=%.6e dpsi=%.6e dy0=%.3e\n", it, Ln,
                       d2, gd, dpsi, dy0);
        if (gd + (1.0 - o.chi) * Ln / 4.0 * d2 >= dpsi - slack) break;
        Ln *= 2.0;
        if (Ln > 1e30) {
          R.fista_failures++;
          *Lout = Ln;
          return false;
        }
      }
      const double A_new = A + a, tk_new = tk + a * mu;            // step 3
      const double snorm = (Ln - mu) * std::sqrt(d2);
      *Lout = Ln;
      // steps 4 and 5 read only scalars of this trial, and x_{j+1} serves
      // only later iterations: an iteration that returns skips its update
      if (dy0 < o.chi * A_new * Ln * d2) {                          // step 4
        R.fista_failures++;
        return false;
      }
      if (snorm <= o.sigma * std::sqrt(dy0)) return true;           // step 5
      // step 3's x update; the next iteration's first trial keeps L = Ln,
      // so its x~ comes out of the same pass
      launch_fista_x_xt(c, x, ynew, xt, mu, a, tk, tk_new, Ln, A_new,
                        next_a(tk_new, A_new, Ln, mu), ld);
      xt_ready = true;
      std::swap(y, ynew);
      A = A_new;
      tk = tk_new;
      L = Ln;
    }
    R.fista_failures++;
    return false;
  }

  // ADAP-AIPP from Ytil; on return Ytil holds W, Wy = (C + A*(p'))W, rY its
  // residual and *gs the operator scalars at W.
  void aipp(double rho, GradScal* gs) {
    copyf(ctr, Ytil);
    grad_enqueue(ctr, nullptr, r_ctr);
    fetch();
    double nrm_ctr2 = c->h_scal[S_PRE];
    for (int j = 0; j < o.max_aipp; ++j) {
      R.aipp_iters++;
      check_time();
      double L = 1.0, VmD2 = 0.0;
      bool stalled = false;
      GradScal gy;
      for (;;) {
        const double Mlow = std::fmax(1.0, Mbar / 2.0);            // step 1
        if (fista(lam, 0.5, Mlow, &L)) {
          grad_enqueue(ynew, Wy, rY);
          change_enqueue(ctr, ynew, r_ctr, nullptr);
          launch_aipp_check(c, Wy, z, ynew, ctr, lam, L, ld);
          fetch();
          gy = grad_read();
          const double dg = change_read(nrm_ctr2);
          const double VD = c->h_scal[S_VEC2];
          const double D2 = c->h_scal[S_VEC2 + 1];
          VmD2 = c->h_scal[S_VEC2 + 2];
          if (o.verbose >= 2)
            std::fprintf(stderr, "[aipp] j=%d lam=%.3e L=%.3e dg=%.6e D2=%.3e VD=%.6e |R|=%.3e rho=%.3e\n",
                         j, lam, L, dg, D2, VD, std::sqrt(VmD2) / lam, rho);
          const double slack = kRoundSlack * unit() * lam * gy.mag;
          stalled = D2 == 0.0;
          if (stalled || -lam * dg - 0.5 * D2 >= -VD - slack) break;  // step 2
        }
        lam /= 2.0;
        if (lam < 1e-30) throw Err{HALLAR_ENUMERIC, "ADAP-AIPP: prox stepsize underflow"};
      }
      Mbar = L;
      const double Rn = std::sqrt(VmD2) / lam;                      // |R_j|, eq. Rj def
      std::swap(ctr, ynew);  // the accepted point is the next prox centre
      std::swap(r_ctr, rY);
      nrm_ctr2 = gy.nrm2;
      // step 3; a prox step that left W unchanged (below the resolution of
      // the stored factor) cannot make further progress: stop there too
      if (Rn <= rho || stalled || j + 1 == o.max_aipp) {
        std::swap(Ytil, ctr);
        std::swap(rY, r_ctr);
        *gs = gy;
        return;
      }
    }
  }

  void trim_rank() {
    // keep the r_cap leading eigenvectors of Y^T Y (Y = Ytil, rank columns)
    const int k = o.r_cap;
    const int ld_new = padded_ld(c, k);
    trim_factor(c, Ytil, ld, rank, k, tmp, ld_new, nullptr);
    std::swap(Ytil, tmp);
    rank = k;
    ld = ld_new;
    R.trims++;
  }

  hallar_status run(const void* U0d, int r0, const double* p0d, hallar_result* out) {
    t0 = std::chrono::steady_clock::now();
    const double tauv = tau();
    // initial factor: padded copy, projected onto the ball
    rank = r0;
    ld = padded_ld(c, r0);
    launch_pad_copy(c, U0d, r0, Ytil, ld, r0, 1.0);
    launch_norm2(c, Ytil, ld, S_VEC);
    if (p0d) HL_CUDA(cudaMemcpyAsync(p, p0d, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    else HL_CUDA(cudaMemsetAsync(p, 0, m * sizeof(double), c->stream));
    refresh_pk();
    fetch();
    const double nU = std::sqrt(c->h_scal[S_VEC]);
    if (nU > tauv) launch_scale(c, Ytil, ld, tauv / nU);
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
    double prev_rnorm = INFINITY;
    bool have_vprev = false;
    grad_enqueue(Ytil, nullptr, nullptr);  // pval at the start point
    fetch();
    double pval_now = grad_read().T0;
    double theta = 0.0, lam_min = 0.0;
    GradScal gs;
    hallar_status st = HALLAR_ENOTCONV;
    for (int t = 1; t <= o.max_outer; ++t) {
      R.outer_iters++;
      const double eps_floor = 0.5 * o.tol * (1.0 + std::fabs(pval_now));
      const double eps_t = std::fmax(eps_floor, eps1 * std::pow(o.eps_decay, t - 1));
      const double rho_t = eps_t / std::fmax(tauv, 1e-300);
      for (int hl = 0; hl < o.max_hlr; ++hl) {                      // HLR
        R.hlr_iters++;
        aipp(rho_t, &gs);                                           // step 6
        launch_dot(c, Wy, Ytil, ld, S_VEC);                         // G . YY^T = <GY, Y>
        launch_axpy_t(c, m, pshift, p, rY, beta);                   // p' = p + beta r(Y)
        const uint64_t sd = o.seed + 7919ull * (uint64_t)R.hlr_iters;
        launch_splitmix(c, sd, v0, 0.1 / std::sqrt((double)n), have_vprev ? vprev : nullptr);
        fetch();
        const double GdotX = c->h_scal[S_VEC];
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
        launch_fw_denom(c, v, rY, theta > 0.0 ? P.tau2 : 0.0, S_VEC2);
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
        if (theta > 0.0) {
          if (alpha >= 1.0) {
            ldn = padded_ld(c, 1);
            launch_fw_append(c, Ytil, ld, 0, v, 0.0, tauv, tmp, ldn, 1);
            rank = 1;
          } else {
            ldn = padded_ld(c, rank + 1);
            launch_fw_append(c, Ytil, ld, rank, v, std::sqrt(1.0 - alpha),
                             std::sqrt(alpha) * tauv, tmp, ldn, 1);
            rank += 1;
          }
        } else if (alpha >= 1.0) {
          ldn = padded_ld(c, 1);
          launch_fw_append(c, Ytil, ld, 0, v, 0.0, 0.0, tmp, ldn, 0);
          rank = 1;
        } else {
          launch_fw_append(c, Ytil, ld, rank, v, std::sqrt(1.0 - alpha), 0.0, tmp, ld, 0);
        }
        ld = ldn;
        std::swap(Ytil, tmp);
        if (rank > o.r_cap) trim_rank();
        check_time();
      }
      // U_t = Y; dual update p_t = p + beta r (step 14)
      launch_axpy_t(c, m, p, p, rY, beta);
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
      // the penalty grows only while primal infeasibility is above the tolerance
      if (rp > o.tol && rnorm > 0.25 * prev_rnorm) beta = std::fmin(2.0 * beta, o.beta_max);
      prev_rnorm = rnorm;
      pval_now = pval;
      check_time();
    }
    sync(c);
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    c->sol_U = Ytil;
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
    keep_buffers();
    s.R.seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - s.t0).count();
    if (res) {
      *res = s.R;
      res->kernel_launches = c->launches - launches0;
    }
    if (e.st == HALLAR_ETIMEOUT && s.Ytil) {
      c->sol_U = s.Ytil;
      c->sol_rank = s.rank;
      c->sol_ld = s.ld;
      c->sol_p = s.p;
    }
    throw;
  }
}

}  // namespace hallar
