// Device-side control of ADAP-AIPP (Appendix A) and ADAP-FISTA (Appendix
// A.1).  The scalar recurrences and tests of both methods run in one-thread
// kernels on the state in a LoopCtl (hallar_internal.cuh), between the
// operator kernels of each trial, so a whole ADAP-AIPP call runs as one CUDA
// graph (an outer WHILE node over ADAP-FISTA calls, an inner WHILE node over
// ADAP-FISTA trials) with no host round trip per trial.  Each control
// kernel writes the arguments of the operator kernels that follow it
// (GradInd, VcInd, ... in the LoopCtl) and sets its loop's condition.
//
// Every loop is bounded on the device: an ADAP-FISTA call stops after
// max_fista iterations or trial_cap trials, the outer loop after
// attempt_cap ADAP-FISTA calls per graph launch (the host then checks the
// time limit and relaunches), and a control kernel always writes its
// condition, so no graph launch can run without end.
//
// The step-2 tests use the same floating-point reading as the oracle:
// g(y) - g(x) formed in difference form by the value-change kernel, and an
// allowance of slack_u * lam * (sum of the magnitudes of g's terms).
#include <cmath>
#include <cstdio>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

namespace {

constexpr int kFistaRunning = 0, kFistaSuccess = 1, kFistaFailure = 2;

__device__ inline void set_cond(unsigned long long h, int graph_mode, int v) {
  if (graph_mode) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v ? 1u : 0u);
}

// step 2's a_j for the trial stepsize Ln: the positive root of
// (Ln - mu) a^2 = tk (A + a)
__device__ inline double next_a(double tk, double A, double Ln, double mu) {
  return (tk + sqrt(tk * tk + 4.0 * tk * A * (Ln - mu))) / (2.0 * (Ln - mu));
}

// a double as the kernels see it (rounded to the factor type)
__device__ inline double as_factor(const LoopCtl& L, double v) {
  return L.mixed ? (double)(float)v : v;
}

// g(Y) - g(X) from the value-change pieces (S_DIFF) and |X|_F^2 (trace row)
__device__ double change_value(const LoopCtl& L, const double* h, double nrmX2) {
  const double dT0 = h[S_DIFF] + (L.C_J != 0.0 ? L.C_J * h[S_DIFF + 9] : 0.0);
  double pd = h[S_DIFF + 1], q = h[S_DIFF + 2];
  if (L.has_trace) {
    const double dt = h[S_DIFF + 3];
    const double rx = nrmX2 - L.b_tr;
    pd += L.p_tr * dt;
    q += dt * (2.0 * rx + dt);
  }
  return dT0 + pd + 0.5 * L.beta * q;
}

// sum of the magnitudes of g's terms at U from the operator's sums (S_GRAD,
// S_PRE): the scale of g's rounding
__device__ double magnitude(const LoopCtl& L, const double* h, double nrm2) {
  double mag = h[S_GRAD + 3] + fabs(L.C_J) * h[S_PRE + 1];
  if (L.has_trace) mag += fabs(L.p_tr + L.beta * (nrm2 - L.b_tr)) * nrm2;
  return mag;
}

// arguments of the next ADAP-FISTA trial at x~ (the centre until x~ has a
// buffer of its own)
__device__ void fill_trial(LoopCtl& L) {
  const void* xt = L.xt_alias ? L.pool[L.i_ctr] : L.xtb;
  const void* ctr = L.pool[L.i_ctr];
  GradInd g;
  g.U = xt;
  g.out = L.zb;
  g.resid = L.rX;
  g.ctr = ctr;
  g.beta = L.beta;
  g.c2lam = 2.0 * L.lam;
  g.invL = 1.0 / L.Ln;
  g.L = L.Ln;
  L.g_trial = g;
  ColInd c;
  c.U = xt;
  L.c_trial = c;
  ColInd cd;
  cd.U = xt;
  cd.Y = L.zb;
  cd.y_from_z = 1;
  L.cd_trial = cd;
  TraceInd t;
  t.dst = L.rX;
  L.t_trial = t;
  VcInd v;
  v.X = xt;
  v.Y = L.zb;
  v.rX = L.rX;
  v.ctr = ctr;
  v.y_out = L.pool[L.i_ynew];
  L.v_trial = v;
}

// arguments of ADAP-AIPP's step-2 evaluation at the ADAP-FISTA output y
__device__ void fill_check(LoopCtl& L, int active) {
  const void* y = L.pool[L.i_ynew];
  const void* ctr = L.pool[L.i_ctr];
  ColInd c;
  c.U = y;
  c.active = active;
  L.c_check = c;
  GradInd g;
  g.U = y;
  g.resid = L.rpool[1 - L.i_rctr];
  g.ctr = ctr;
  g.zin = L.zb;
  g.beta = L.beta;
  g.c2lam = 2.0 * L.lam;
  g.L = L.Lacc;
  g.active = active;
  L.g_check = g;
  TraceInd t;
  t.dst = L.rpool[1 - L.i_rctr];
  t.active = active;
  L.t_check = t;
  ColInd cd;
  cd.U = ctr;
  cd.Y = y;
  cd.active = active;
  L.cd_check = cd;
  VcInd v;
  v.X = ctr;
  v.Y = y;
  v.rX = L.rpool[L.i_rctr];
  v.active = active;
  L.v_check = v;
}

__global__ void k_loop_reset(LoopCtl* Lp) {
  if (threadIdx.x == 0 && blockIdx.x == 0) Lp->attempts = 0;
}

// ADAP-AIPP step 1: an ADAP-FISTA call from x_0 = W_{j-1} (the centre) with
// M_j = max(1, Mbar_{j-1} / 2)
__global__ void k_aipp_begin(LoopCtl* Lp) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  LoopCtl& L = *Lp;
  if (L.error || L.done) {
    L.fista_status = kFistaFailure;
    L.xi.active = 0;
    L.g_trial.active = L.v_trial.active = L.c_trial.active = L.cd_trial.active = 0;
    L.t_trial.active = 0;
    fill_check(L, 0);
    L.cont_fista = 0;
    set_cond(L.h_fista, L.graph_mode, 0);
    return;
  }
  L.A = 0.0;
  L.tk = 1.0;
  L.L = fmax(1.0, L.Mbar / 2.0);
  L.Ln = L.L;
  L.a = next_a(L.tk, L.A, L.Ln, L.mu);
  L.fista_it = 0;
  L.fista_status = kFistaRunning;
  L.trials = 0;
  L.x_alias = 1;
  L.xt_alias = 1;
  L.i_y = L.i_ctr;
  L.i_ynew = (L.i_ctr + 1) % 3;
  L.xi.active = 0;
  L.n_fista_iters++;
  fill_trial(L);
  L.cont_fista = 1;
  set_cond(L.h_fista, L.graph_mode, 1);
}

// ADAP-FISTA after a trial (the operator sums in h): step 2's test, then
// steps 3-5 for an accepted trial
__global__ void k_fista_ctl(LoopCtl* Lp, const double* __restrict__ h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  LoopCtl& L = *Lp;
  int cont = 0;
  L.trials++;
  L.n_trials++;
  L.n_grads++;
  L.n_values++;
  if (L.error == 0 && L.fista_status == kFistaRunning) {
    const double nrm_xt2 = h[S_PRE];
    const double invL = as_factor(L, 1.0 / L.Ln);
    // <grad psi_s(x~), y - x~> = <x~ - z, y - x~> / invL (z = x~ - g invL),
    // reduced from the vectors by the value change
    const double gd = h[S_DIFF + 7] / invL;
    const double d2 = h[S_DIFF + 4], dlin = h[S_DIFF + 5], dy0 = h[S_DIFF + 6];
    const double dpsi = L.lam * change_value(L, h, nrm_xt2) + dlin;
    const double slack = L.slack_u * L.lam * magnitude(L, h, nrm_xt2);
    if (!isfinite(dpsi) || !isfinite(gd)) {
      L.error = HALLAR_ENUMERIC;
    } else if (gd + (1.0 - L.chi) * L.Ln / 4.0 * d2 >= dpsi - slack) {
      // step 3
      const double A_new = L.A + L.a, tk_new = L.tk + L.a * L.mu;
      const double snorm = (L.Ln - L.mu) * sqrt(d2);
      L.Lacc = L.Ln;
      // y equal to x_0 within rounding: x_0 is the prox point to working
      // precision and step 4 would compare rounding-level numbers (the
      // oracle's reading); the call succeeds
      const bool at_x0 = dy0 <= L.slack_u * L.slack_u * L.nrm_ctr2;
      if (!at_x0 && dy0 < L.chi * A_new * L.Ln * d2) {            // step 4
        L.fista_status = kFistaFailure;
        L.n_fista_fail++;
        if (L.verbose >= 3)
          printf("[fista4] it=%d lam=%.6e dy0=%.9e A=%.9e Ln=%.9e d2=%.9e\n", L.fista_it,
                 L.lam, dy0, A_new, L.Ln, d2);
      } else if (at_x0 || snorm <= L.sigma * sqrt(dy0)) {         // step 5
        L.fista_status = kFistaSuccess;
      } else if (L.fista_it + 1 >= L.max_fista) {
        L.fista_status = kFistaFailure;
        L.n_fista_fail++;
        if (L.verbose >= 3) printf("[fista-max] lam=%.6e\n", L.lam);
      } else {
        // step 3's x update and the next iteration's first x~ (whose
        // stepsize is the accepted Ln) in one pass after this kernel
        const double a_next = next_a(tk_new, A_new, L.Ln, L.mu);
        const int iy = L.i_ynew;
        XInd x;
        x.mode = 1;
        x.active = 1;
        x.x = L.xb;
        x.x_src = L.x_alias ? L.pool[L.i_ctr] : L.xb;
        x.xt = L.xtb;
        x.xt_src = L.xt_alias ? L.pool[L.i_ctr] : L.xtb;
        x.y = L.pool[iy];
        x.c0 = (L.mu * L.a + L.a * (L.Ln - L.mu)) / tk_new;
        x.c1 = L.tk / tk_new;
        x.c2 = -L.a * (L.Ln - L.mu) / tk_new;
        x.w0 = A_new / (A_new + a_next);
        x.w1 = a_next / (A_new + a_next);
        L.xi = x;
        L.x_alias = 0;
        L.xt_alias = 0;
        L.i_y = iy;
        L.i_ynew = 3 - L.i_ctr - iy;
        L.A = A_new;
        L.tk = tk_new;
        L.L = L.Ln;
        L.a = a_next;
        L.fista_it++;
        L.n_fista_iters++;
        fill_trial(L);
        cont = 1;
      }
    } else {
      // step 2 rejects: double L and retry with a new x~
      L.Ln *= 2.0;
      if (L.Ln > 1e30) {
        L.fista_status = kFistaFailure;
        L.n_fista_fail++;
      } else {
        L.a = next_a(L.tk, L.A, L.Ln, L.mu);
        if (L.A > 0.0) {
          XInd x;
          x.mode = 0;
          x.active = 1;
          x.xt = L.xtb;
          x.x_src = L.x_alias ? L.pool[L.i_ctr] : L.xb;
          x.y = L.pool[L.i_y];
          x.w0 = L.A / (L.A + L.a);
          x.w1 = L.a / (L.A + L.a);
          L.xi = x;
          L.xt_alias = 0;
        } else {
          L.xi.active = 0;  // x~ = x_0 = the centre for every L
        }
        fill_trial(L);
        cont = 1;
      }
    }
  }
  if (cont && L.trials >= L.trial_cap) {
    L.error = HALLAR_ENOTCONV;
    cont = 0;
  }
  if (!cont) {
    L.xi.active = 0;
    if (L.fista_status == kFistaRunning) L.fista_status = kFistaFailure;
    fill_check(L, L.fista_status == kFistaSuccess && L.error == 0);
  }
  L.cont_fista = cont;
  set_cond(L.h_fista, L.graph_mode, cont);
}

// ADAP-AIPP after an ADAP-FISTA call: step 2's inequality (evaluated at the
// ADAP-FISTA output y), acceptance as W_j (step 3's residual test) or a
// halved prox stepsize
__global__ void k_aipp_ctl(LoopCtl* Lp, const double* __restrict__ h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  LoopCtl& L = *Lp;
  L.attempts++;
  L.n_attempts++;
  if (L.error == 0 && !L.done) {
    bool accept = false, stalled = false;
    double nrm_y2 = 0.0, VmD2 = 0.0;
    if (L.fista_status == kFistaSuccess) {
      L.n_grads++;
      L.n_values++;
      nrm_y2 = h[S_PRE];
      const double mag = magnitude(L, h, nrm_y2);
      const double VD = h[S_GRAD + 4], D2 = h[S_GRAD + 5];
      VmD2 = h[S_GRAD + 6];
      const double dg = change_value(L, h, L.nrm_ctr2);
      const double slack = L.slack_u * L.lam * mag;
      stalled = D2 == 0.0;
      accept = stalled || -L.lam * dg - 0.5 * D2 >= -VD - slack;
      if (L.verbose >= 3)
        printf("[aipp2] j=%d lam=%.6e dg=%.9e D2=%.9e VD=%.9e slack=%.9e mag=%.9e %s\n",
               L.aipp_j, L.lam, dg, D2, VD, slack, mag, accept ? "accept" : "reject");
      if (accept) {
        double T0 = h[S_GRAD] + L.C_J * h[S_PRE + 1];
        double pr = h[S_GRAD + 1], rr = h[S_GRAD + 2];
        if (L.has_trace) {
          const double rt = nrm_y2 - L.b_tr;
          pr += L.p_tr * rt;
          rr += rt * rt;
        }
        L.gT0 = T0;
        L.gpr = pr;
        L.grr = rr;
        L.gmag = mag;
        L.gnrm2 = nrm_y2;
        L.gWU = h[S_GRAD + 7];
      }
    }
    if (accept) {
      L.Mbar = L.Lacc;
      L.Rn = sqrt(VmD2) / L.lam;                  // |R_j|, eq. Rj def
      L.i_ctr = L.i_ynew;                         // W_j is the next centre
      L.i_rctr = 1 - L.i_rctr;
      L.nrm_ctr2 = nrm_y2;
      L.aipp_j++;
      L.n_aipp_iters++;
      // step 3; a prox step that left W unchanged cannot make progress
      if (L.Rn <= L.rho || stalled || L.aipp_j >= L.max_aipp) L.done = 1;
      L.stall_exit = stalled;
    } else {
      L.lam /= 2.0;
      if (L.lam < 1e-30) L.error = HALLAR_ENUMERIC;
    }
  }
  const int cont = !(L.done || L.error) && L.attempts < L.attempt_cap;
  L.cont_aipp = cont;
  set_cond(L.h_aipp, L.graph_mode, cont);
}

// ADAP-FISTA's x and x~ updates (XInd): mode 0 x~ = w0 y + w1 x; mode 1
// x <- c0 y + c1 x + c2 x~, then x~ = w0 y + w1 x (the same arithmetic, in
// the factor type, as the host-driven passes)
template <class T>
__global__ void __launch_bounds__(kBlock) k_loop_x(int64_t nvec, const LoopCtl* __restrict__ Lp) {
  const XInd s = Lp->xi;
  if (!s.active) return;
  constexpr int VEC = V16<T>::N;
  const T* y = static_cast<const T*>(s.y);
  const T* xs = static_cast<const T*>(s.x_src);
  // coefficients in the factor type, converted by one thread of the block
  __shared__ T s_c[5];
  if (threadIdx.x == 0) {
    s_c[0] = (T)s.w0;
    s_c[1] = (T)s.w1;
    s_c[2] = (T)s.c0;
    s_c[3] = (T)s.c1;
    s_c[4] = (T)s.c2;
  }
  __syncthreads();
  const T w0 = s_c[0], w1 = s_c[1];
  T* xt = static_cast<T*>(s.xt);
  if (s.mode == 0) {
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < nvec;
         v += (int64_t)gridDim.x * kBlock) {
      T a[VEC], b[VEC], o[VEC];
      load_chunk<T>(y, v * VEC, a);
      load_chunk<T>(xs, v * VEC, b);
#pragma unroll
      for (int k = 0; k < VEC; ++k) o[k] = tfma(w0, a[k], w1 * b[k]);
      store_chunk<T>(xt, v * VEC, o);
    }
  } else {
    const T* xts = static_cast<const T*>(s.xt_src);
    T* x = static_cast<T*>(s.x);
    const T c0 = s_c[2], c1 = s_c[3], c2 = s_c[4];
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < nvec;
         v += (int64_t)gridDim.x * kBlock) {
      T a[VEC], b[VEC], t[VEC], o[VEC], q[VEC];
      load_chunk<T>(y, v * VEC, a);
      load_chunk<T>(xs, v * VEC, b);
      load_chunk<T>(xts, v * VEC, t);
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        o[k] = tfma(c0, a[k], tfma(c1, b[k], c2 * t[k]));
        q[k] = tfma(w0, a[k], w1 * o[k]);
      }
      store_chunk<T>(x, v * VEC, o);
      store_chunk<T>(xt, v * VEC, q);
    }
  }
}

// trace-row residual entry from the pre-pass's |U|_F^2: dst[m-1] = *dscal + add
template <class T>
__global__ void k_trace_fix_ind(const TraceInd* __restrict__ ti, int64_t m,
                                const double* __restrict__ dscal, double add) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const TraceInd t = *ti;
  if (!t.active) return;
  static_cast<T*>(t.dst)[m - 1] = (T)(dscal[0] + add);
}

}  // namespace

void launch_loop_reset(Ctx* c, LoopCtl* L) {
  k_loop_reset<<<1, 32, 0, c->stream>>>(L);
  HL_CHECK_LAUNCH(c);
}

void launch_aipp_begin(Ctx* c, LoopCtl* L) {
  k_aipp_begin<<<1, 32, 0, c->stream>>>(L);
  HL_CHECK_LAUNCH(c);
}

void launch_fista_ctl(Ctx* c, LoopCtl* L) {
  k_fista_ctl<<<1, 32, 0, c->stream>>>(L, c->d_scal);
  HL_CHECK_LAUNCH(c);
}

void launch_aipp_ctl(Ctx* c, LoopCtl* L) {
  k_aipp_ctl<<<1, 32, 0, c->stream>>>(L, c->d_scal);
  HL_CHECK_LAUNCH(c);
}

void launch_loop_x(Ctx* c, int ld, LoopCtl* L) {
  const bool mixed = c->opt.precision == HALLAR_MIXED;
  const int vec = mixed ? V16<float>::N : V16<double>::N;
  const int64_t nvec = c->P.n * (int64_t)ld / vec;
  if (mixed) {
    const int grid = wave_grid(c, k_loop_x<float>, nvec, kBlock * 4, kBlock);
    k_loop_x<float><<<grid, kBlock, 0, c->stream>>>(nvec, L);
  } else {
    const int grid = wave_grid(c, k_loop_x<double>, nvec, kBlock * 4, kBlock);
    k_loop_x<double><<<grid, kBlock, 0, c->stream>>>(nvec, L);
  }
  HL_CHECK_LAUNCH(c);
}

void launch_trace_fix_ind(Ctx* c, const TraceInd* ti, double add) {
  if (c->opt.precision == HALLAR_MIXED)
    k_trace_fix_ind<float><<<1, 32, 0, c->stream>>>(ti, c->P.m, c->d_scal + S_PRE, add);
  else
    k_trace_fix_ind<double><<<1, 32, 0, c->stream>>>(ti, c->P.m, c->d_scal + S_PRE, add);
  HL_CHECK_LAUNCH(c);
}

}  // namespace hallar
