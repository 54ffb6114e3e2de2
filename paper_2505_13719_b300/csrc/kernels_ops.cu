// Operator kernels of the HALLaR hot path on the n x r factor U.
//
// k_grad fuses, in one pass over the merged CSR, the constraint map
// T = A~(UU^T) (Section 4.1, eq. A tilde operator; the sum Alg. 2 computes),
// the multiplier shift p' = p + beta (A(UU^T) - b) and the SpMM
// W = (C + A*(p'))U (Section 4.2, eq. Adjoint calculation; Alg. 4 forms M and
// multiplies): each row gathers its neighbour rows once, forms the row dot
// products it needs, shifts the multipliers in registers and accumulates W.
// M is never stored.
//
// Thread mapping: a group of G lanes owns one row; lane l of the group holds
// the 16-byte chunks l, l+G, ... of the row (K chunks), so every row access is
// a 128-bit vector load and a group reads a 256-byte FP64 row (r = 32) with
// one instruction per lane.  Gathered neighbour rows are read through L1
// (ld.global.nc): on mesh-like graphs neighbours i +- 1 are rows of the same
// warp or block, and the rest of the gather window of a row-ordered sweep
// sits in the 126 MB L2.
#include <cmath>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

namespace {

// Resident blocks per SM the register allocation must allow, for the float
// diagonal-family kernels with one thread per row of up to three 16-byte
// chunks (Max-Cut in the mixed form): each thread keeps one row's gathers in
// flight, so more warps hide more latency.  `want` is 4 (64 registers) for
// the plain passes and 3 (80 registers) for the variants with the most live
// sums; every other shape keeps the compiler's own register count.
template <class T, int FAM, int G, int K, int want>
constexpr int kMinBlocks =
    (sizeof(T) == 4 && FAM == FAM_DIAG && G == 1 && K <= 3) ? want : 1;

// edges whose metadata one group loads at once (at most the group's lanes)
template <int G>
constexpr int kEdgeBatch = G < 4 ? G : 4;

template <int FAM>
struct FamTraits {
  static constexpr bool kDiag = FAM == FAM_DIAG;
  static constexpr bool kPairs = FAM != FAM_DIAG;
  static constexpr bool kCval = FAM != FAM_EDGE;
};

// Per-row vectors (b, p, the diagonal of C, residuals) have the factor's
// element type T: the float form reads float copies and keeps every per-row
// operation in float (see Acc in device_common.cuh); the grid reductions are
// double.
struct OpArgs {
  int64_t n;
  int ld;
  const int* __restrict__ rowptr;
  const int* __restrict__ col;
  const int* __restrict__ code;
  const void* __restrict__ cval;      // T
  const void* __restrict__ cdiag;     // T
  const void* __restrict__ b;         // T
  const void* __restrict__ p;         // T
  double C_J;
  double beta;
  int has_trace;
  int64_t trace_row;
  double* partials;
  unsigned* counter;
  double* out;
};

// ---------------------------------------------------------------------------
// fused constraint map + shift + SpMM
// ---------------------------------------------------------------------------
struct GradIO {
  const void* __restrict__ cjv;       // T[ld] or null: C_J 11^T U = 1 (C_J colsum)^T
  const double* __restrict__ pre;     // pre[0] = |U|_F^2 (trace row)
  void* __restrict__ Tout;            // T: A_l . UU^T at [l], or null
};

// Epilogues of the row pass (what the kernel does with W_i = (C + A*(p'))_i U
// once row i is complete; W itself is formed in registers):
//   EPI_W        store W (hallar_grad, the outer loop)
//   EPI_FISTA_Z  ADAP-FISTA step 2's unprojected step at U = x~ (Appendix A.1):
//                g = grad psi_s(x~) = 2 lam W + x~ - centre, z = x~ - g / L;
//                store z; reduce |z|^2 (the ball projection's factor
//                min(1, tau/|z|); the value change that forms y = P_B(z)
//                reduces <g, y - x~>)
//   EPI_AIPP     ADAP-AIPP step 2 at U = y (z its unprojected step):
//                V - D = 2 lam W + L (z - y), D = y - centre; reduce <V, D>,
//                |D|^2, |V - D|^2 (R_j = (V - D)/lam, eq. Rj def) and <W, y>
//                (G . YY^T of the gap test); W is not stored
// The pointers and coefficients come from a GradInd, by value or (when the
// device-side ADAP-AIPP loop fills it) from device memory.
template <int EPI>
constexpr int kGradRed = EPI == EPI_W ? 4 : (EPI == EPI_FISTA_Z ? 5 : 8);

// CJ: C has the implicit C_J 11^T part (a compile-time switch: an unused
// runtime branch would still cost predicated instructions in the row loop)
template <class T, int FAM, int G, int K, bool CJ, int EPI>
__global__ void __launch_bounds__(kBlock, kMinBlocks<T, FAM, G, K, EPI == EPI_W ? 4 : 3>) k_grad(OpArgs a, GradIO io, GradInd gi,
                                                 const GradInd* __restrict__ gind) {
  using Tr = FamTraits<FAM>;
  constexpr int VEC = V16<T>::N;
  if (gind != nullptr) gi = *gind;
  if (!gi.active) return;  // uniform over the grid: no block reaches the reduction
  const T* __restrict__ U = static_cast<const T*>(gi.U);
  const T* __restrict__ cval = static_cast<const T*>(a.cval);
  const T* __restrict__ cdiag = static_cast<const T*>(a.cdiag);
  const T* __restrict__ bv = static_cast<const T*>(a.b);
  const T* __restrict__ pv = static_cast<const T*>(a.p);
  T* __restrict__ W = static_cast<T*>(gi.out);
  T* __restrict__ resid = static_cast<T*>(gi.resid);
  T* __restrict__ Tout = static_cast<T*>(io.Tout);
  const T* __restrict__ cjv = static_cast<const T*>(io.cjv);
  const T* __restrict__ ctr = static_cast<const T*>(gi.ctr);
  const T* __restrict__ zin = static_cast<const T*>(gi.zin);
  const int lane_g = threadIdx.x & (G - 1);
  const unsigned gmask = group_mask<G>();
  const int64_t ngroups = (int64_t)gridDim.x * (kBlock / G);
  const int nch = a.ld / VEC;
  // coefficients in the factor type and the trace row's shifted multiplier
  // (identical for every row), formed by one thread of the block: double
  // arithmetic and conversions occupy the slow FP64 pipe
  __shared__ T s_coef[5];
  if (threadIdx.x == 0) {
    s_coef[0] = (T)gi.beta;
    s_coef[1] = (T)gi.c2lam;
    s_coef[2] = (T)gi.invL;
    s_coef[3] = (T)gi.L;
    T pst = (T)0;
    if (Tr::kPairs && a.has_trace) {
      const double rt = io.pre[0] - (double)bv[a.trace_row];
      pst = (T)((double)pv[a.trace_row] + gi.beta * rt);
    }
    s_coef[4] = pst;
  }
  __syncthreads();
  const T beta = s_coef[0];
  const T c2lam = s_coef[1], invL = s_coef[2], Lt = s_coef[3];
  const T ps_tr = s_coef[4];

  // C.UU^T (sparse + diagonal part), p.r, r.r, and the magnitude
  // sum |p'_l| |A_l.UU^T| + |C terms| that scales the rounding of g;
  // e0..e3: the epilogue's sums
  Acc<T> acc_t0, acc_pr, acc_rr, acc_mag, e0s, e1s, e2s, e3s;
  // the next row's entry range is loaded one iteration ahead, so a row's
  // column loads need not wait for its row pointers
  int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / G;
  int e0n = 0, e1n = 0;
  if (i < a.n) {
    e0n = a.rowptr[i];
    e1n = a.rowptr[i + 1];
  }
  for (; i < a.n; i += ngroups) {
    const int e0 = e0n, e1 = e1n;
    if (i + ngroups < a.n) {
      e0n = a.rowptr[i + ngroups];
      e1n = a.rowptr[i + ngroups + 1];
    }
    T u[K][VEC], acc[K][VEC];
    const int64_t rowoff = i * (int64_t)a.ld;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int ch = lane_g + k * G;
      if (ch < nch) {
        load_chunk<T>(U, rowoff + ch * VEC, u[k]);
      } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) u[k][v] = (T)0;
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[k][v] = (T)0;
    }
    T nrm_l = (T)0;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int v = 0; v < VEC; ++v) nrm_l = tfma(u[k][v], u[k][v], nrm_l);
    const T nrm = group_sum<G>(nrm_l, gmask);  // |U_i|^2

    const T cdi = cdiag[i];
    T dcoef = cdi;
    if (Tr::kDiag) {
      // constraint i: A_i . UU^T = |U_i|^2
      const T r = nrm - bv[i];
      const T pi = pv[i];
      const T ps = tfma(beta, r, pi);
      dcoef += ps;
      if (lane_g == 0) {
        acc_pr.add(pi * r);
        acc_rr.add(r * r);
        acc_mag.add(tabs(ps) * nrm);
        if (resid) resid[i] = r;
        if (Tout) Tout[i] = nrm;
      }
    }
    if (Tr::kPairs) dcoef += ps_tr;

    T cdot_l = (T)0;  // lane part of <U_i, sum_j C_ij U_j> over the C entries
    // one merged entry (column j, C value cv, constraint code cd) with the
    // gathered row U_j
    auto apply_edge = [&](const T (&uj)[K][VEC], T cv, int cd) {
      T coef;
      bool is_c;
      if (Tr::kDiag) {
        coef = cv;
        is_c = true;
      } else {
        is_c = Tr::kCval && cd == kNoCons;
        if (is_c) {
          coef = cv;
        } else {
          // pair constraint l: A_l . UU^T = <U_i, U_j>
          T d_l = (T)0;
#pragma unroll
          for (int k = 0; k < K; ++k)
#pragma unroll
            for (int v = 0; v < VEC; ++v) d_l = tfma(u[k][v], uj[k][v], d_l);
          const T dot = group_sum<G>(d_l, gmask);
          const bool owner = cd >= 0;
          const int l = owner ? cd : -cd - 1;
          const T r = dot - bv[l];
          const T pl = pv[l];
          const T ps = tfma(beta, r, pl);
          coef = (T)0.5 * ps;
          if (owner && lane_g == 0) {
            acc_pr.add(pl * r);
            acc_rr.add(r * r);
            acc_mag.add(tabs(ps) * tabs(dot));
            if (resid) resid[l] = r;
            if (Tout) Tout[l] = dot;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          // (diagonal family: acc holds only C terms; its dot with U_i is
          // taken once after the loop)
          if (!Tr::kDiag && is_c) cdot_l = tfma(coef * u[k][v], uj[k][v], cdot_l);
          acc[k][v] = tfma(coef, uj[k][v], acc[k][v]);
        }
    };
    auto gather = [&](int64_t j, T (&uj)[K][VEC]) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int ch = lane_g + k * G;
        if (ch < nch) {
          load_chunk<T>(U, j * a.ld + ch * VEC, uj[k]);
        } else {
#pragma unroll
          for (int v = 0; v < VEC; ++v) uj[k][v] = (T)0;
        }
      }
    };
    if constexpr (G == 1) {
      // one thread per row: entries two at a time, both gathers issued before
      // either is used, so a row's chain of dependent loads is half as long
      int e = e0;
      for (; e + 2 <= e1; e += 2) {
        const int64_t j0 = a.col[e], j1 = a.col[e + 1];
        const T cv0 = Tr::kCval ? cval[e] : (T)0, cv1 = Tr::kCval ? cval[e + 1] : (T)0;
        const int cd0 = Tr::kPairs ? a.code[e] : 0, cd1 = Tr::kPairs ? a.code[e + 1] : 0;
        T uj0[K][VEC], uj1[K][VEC];
        gather(j0, uj0);
        gather(j1, uj1);
        apply_edge(uj0, cv0, cd0);
        apply_edge(uj1, cv1, cd1);
      }
      if (e < e1) {
        T uj0[K][VEC];
        gather(a.col[e], uj0);
        apply_edge(uj0, Tr::kCval ? cval[e] : (T)0, Tr::kPairs ? a.code[e] : 0);
      }
    } else {
      // Edges go in batches: lane t of the group loads the column, value and
      // code of edge eb + t with one instruction and a shuffle hands them to
      // the group, so a row's metadata costs one load round trip per batch
      // instead of one per edge ahead of each gather.
      for (int eb = e0; eb < e1; eb += kEdgeBatch<G>) {
        const int cnt = min(kEdgeBatch<G>, e1 - eb);
        int col_t = 0, code_t = 0;
        T cv_t = (T)0;
        if (lane_g < cnt) {
          col_t = a.col[eb + lane_g];
          if (Tr::kCval) cv_t = cval[eb + lane_g];
          if (Tr::kPairs) code_t = a.code[eb + lane_g];
        }
#pragma unroll
        for (int t = 0; t < kEdgeBatch<G>; ++t) {
          const T cv = Tr::kCval ? group_bcast<G>(cv_t, t, gmask) : (T)0;
          const int cd = Tr::kPairs ? group_bcast<G>(code_t, t, gmask) : 0;
          const int64_t j = group_bcast<G>(col_t, t, gmask);
          if (t >= cnt) continue;  // uniform over the group
          T uj[K][VEC];
          gather(j, uj);
          apply_edge(uj, cv, cd);
        }
      }
    }
    if (Tr::kDiag) {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int v = 0; v < VEC; ++v) cdot_l = tfma(u[k][v], acc[k][v], cdot_l);
    }
    if (lane_g == 0) {
      acc_t0.add(cdot_l + cdi * nrm);
      acc_mag.add(tabs(cdot_l) + tabs(cdi) * nrm);
    } else {
      acc_t0.add(cdot_l);
      acc_mag.add(tabs(cdot_l));
    }

    // the epilogue's sums of this row, added to the compensated
    // accumulators once per row
    T rs0 = (T)0, rs1 = (T)0, rs2 = (T)0, rs3 = (T)0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int ch = lane_g + k * G;
      if (ch >= nch) continue;
      T w[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) w[v] = tfma(dcoef, u[k][v], acc[k][v]);
      if constexpr (CJ) {
        // the C_J 11^T U term adds C_J * colsum to every row of W
#pragma unroll
        for (int v = 0; v < VEC; ++v) w[v] += __ldg(&cjv[ch * VEC + v]);
      }
      if constexpr (EPI == EPI_W) {
        if (W != nullptr) store_chunk<T>(W, rowoff + ch * VEC, w);
      } else if constexpr (EPI == EPI_FISTA_Z) {
        T cc[VEC], zz[VEC];
        load_chunk<T>(ctr, rowoff + ch * VEC, cc);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const T g = tfma(c2lam, w[v], u[k][v] - cc[v]);
          zz[v] = tfma(-invL, g, u[k][v]);
          rs0 = tfma(zz[v], zz[v], rs0);
        }
        store_chunk<T>(W, rowoff + ch * VEC, zz);
      } else {
        T cc[VEC], zz[VEC];
        load_chunk<T>(ctr, rowoff + ch * VEC, cc);
        load_chunk<T>(zin, rowoff + ch * VEC, zz);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const T D = u[k][v] - cc[v];
          const T VmD = tfma(c2lam, w[v], Lt * (zz[v] - u[k][v]));
          rs0 = tfma(VmD + D, D, rs0);
          rs1 = tfma(D, D, rs1);
          rs2 = tfma(VmD, VmD, rs2);
          rs3 = tfma(w[v], u[k][v], rs3);
        }
      }
    }
    if constexpr (EPI != EPI_W) e0s.add(rs0);
    if constexpr (EPI == EPI_AIPP) {
      e1s.add(rs1);
      e2s.add(rs2);
      e3s.add(rs3);
    }
  }
  if constexpr (EPI == EPI_W) {
    Acc<T> red[4] = {acc_t0, acc_pr, acc_rr, acc_mag};
    grid_reduce_acc<T, 4>(red, a.partials, a.counter, a.out);
  } else if constexpr (EPI == EPI_FISTA_Z) {
    Acc<T> red[5] = {acc_t0, acc_pr, acc_rr, acc_mag, e0s};
    grid_reduce_acc<T, 5>(red, a.partials, a.counter, a.out);
  } else {
    Acc<T> red[8] = {acc_t0, acc_pr, acc_rr, acc_mag, e0s, e1s, e2s, e3s};
    grid_reduce_acc<T, 8>(red, a.partials, a.counter, a.out);
  }
}

// ---------------------------------------------------------------------------
// g(Y) - g(X) without cancellation: every pair product difference is
// <Y_a,Y_b> - <X_a,X_b> = <D_a, Y_b> + <X_a, D_b>, D = Y - X.
// YZ: Y = cs Z with cs = min(1, tau/|Z|_F) read from the device (ADAP-FISTA
// step 2's projection onto the ball B_tau, eq. dimensional ball), formed in
// registers for the own row and every gathered neighbour and stored once;
// the pass then also reduces |Y - X|^2, <Y - X, (Y + X)/2 - centre> and
// |Y - centre|^2 (the prox terms of psi_s and step 4's |y - x_0|^2).
// ---------------------------------------------------------------------------
struct DiffIO {
  const double* __restrict__ z2;  // YZ: |Z|_F^2 on the device
  double tau;                     // YZ: the ball radius
};

template <bool YZ>
constexpr int kDiffRed = YZ ? 8 : 4;

template <class T, int FAM, int G, int K, bool YZ>
__global__ void __launch_bounds__(kBlock, kMinBlocks<T, FAM, G, K, 3>) k_value_change(OpArgs a, DiffIO io, VcInd vi,
                                                         const VcInd* __restrict__ vind) {
  using Tr = FamTraits<FAM>;
  constexpr int VEC = V16<T>::N;
  if (vind != nullptr) vi = *vind;
  if (!vi.active) return;  // uniform over the grid
  const T* __restrict__ X = static_cast<const T*>(vi.X);
  const T* __restrict__ Yv = static_cast<const T*>(vi.Y);
  const T* __restrict__ rXv = static_cast<const T*>(vi.rX);
  T* __restrict__ rYv = static_cast<T*>(vi.rY);
  const T* __restrict__ ctr = static_cast<const T*>(vi.ctr);
  T* __restrict__ yout = static_cast<T*>(vi.y_out);
  const T* __restrict__ cval = static_cast<const T*>(a.cval);
  const T* __restrict__ cdiag = static_cast<const T*>(a.cdiag);
  const T* __restrict__ pv = static_cast<const T*>(a.p);
  const int lane_g = threadIdx.x & (G - 1);
  const unsigned gmask = group_mask<G>();
  const int64_t ngroups = (int64_t)gridDim.x * (kBlock / G);
  const int nch = a.ld / VEC;
  // the ball projection's factor, formed by one thread of the block
  __shared__ T s_cs;
  if constexpr (YZ) {
    if (threadIdx.x == 0) {
      const double zn = sqrt(*io.z2);
      s_cs = (T)(zn > io.tau ? io.tau / zn : 1.0);
    }
    __syncthreads();
  }
  const T cs = YZ ? s_cs : (T)1;

  // dT0 (sparse + diagonal part), p.dT, dT (2 rX + dT), trace dT; YZ:
  // |D|^2, <D, (Y + X)/2 - centre>, |Y - centre|^2 and <X - Z, D> (with
  // Z = X - g/L this is <g, Y - X>/L, ADAP-FISTA step 2's linear term, taken
  // from the vectors themselves: formed from <g, X> and |g|^2 it cancels
  // catastrophically when the projection undoes a radial step)
  Acc<T> acc_t0, acc_pd, acc_q, acc_tr, e0s, e1s, e2s, e3s;
  // the next row's entry range is loaded one iteration ahead, so a row's
  // column loads need not wait for its row pointers
  int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / G;
  int e0n = 0, e1n = 0;
  if (i < a.n) {
    e0n = a.rowptr[i];
    e1n = a.rowptr[i + 1];
  }
  for (; i < a.n; i += ngroups) {
    const int e0 = e0n, e1 = e1n;
    if (i + ngroups < a.n) {
      e0n = a.rowptr[i + ngroups];
      e1n = a.rowptr[i + ngroups + 1];
    }
    T x[K][VEC], d[K][VEC];
    const int64_t rowoff = i * (int64_t)a.ld;
    T rs0 = (T)0, rs1 = (T)0, rs2 = (T)0, rs3 = (T)0;  // YZ: this row's prox sums
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int ch = lane_g + k * G;
      T y[VEC];
      if (ch < nch) {
        load_chunk<T>(X, rowoff + ch * VEC, x[k]);
        load_chunk<T>(Yv, rowoff + ch * VEC, y);
        if constexpr (YZ) {
          T cc[VEC];
          load_chunk<T>(ctr, rowoff + ch * VEC, cc);
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const T zv = y[v];
            y[v] = cs * zv;
            const T dd = y[v] - x[k][v];
            const T yc = y[v] - cc[v];
            rs0 = tfma(dd, dd, rs0);
            rs1 = tfma(dd, (T)0.5 * (y[v] + x[k][v]) - cc[v], rs1);
            rs2 = tfma(yc, yc, rs2);
            rs3 = tfma(x[k][v] - zv, dd, rs3);
          }
          store_chunk<T>(yout, rowoff + ch * VEC, y);
        }
      } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) x[k][v] = y[v] = (T)0;
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) d[k][v] = y[v] - x[k][v];
    }
    // <D_i, Y_i + X_i> = <D_i, D_i + 2 X_i> = |Y_i|^2 - |X_i|^2
    T own_l = (T)0;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int v = 0; v < VEC; ++v) own_l = tfma(d[k][v], d[k][v] + (T)2 * x[k][v], own_l);
    if constexpr (YZ) {
      e0s.add(rs0);
      e1s.add(rs1);
      e2s.add(rs2);
      e3s.add(rs3);
    }
    acc_tr.add(own_l);               // trace row change (lane parts)
    if (Tr::kDiag) {
      const T dt = group_sum<G>(own_l, gmask);
      if (lane_g == 0) {
        const T rx = rXv[i];
        acc_pd.add(pv[i] * dt);
        acc_q.add(dt * ((T)2 * rx + dt));
        if (rYv) rYv[i] = rx + dt;
      }
    }
    T cd_l = (T)0;
    // gathered rows X_j and Y_j (Y_j = cs Z_j in the YZ form)
    auto gather = [&](int64_t j, T (&xj)[K][VEC], T (&yj)[K][VEC]) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int ch = lane_g + k * G;
        if (ch < nch) {
          load_chunk<T>(X, j * a.ld + ch * VEC, xj[k]);
          load_chunk<T>(Yv, j * a.ld + ch * VEC, yj[k]);
          if constexpr (YZ) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) yj[k][v] = cs * yj[k][v];
          }
        } else {
#pragma unroll
          for (int v = 0; v < VEC; ++v) xj[k][v] = yj[k][v] = (T)0;
        }
      }
    };
    // one merged entry: <D_i, Y_j> + <X_i, D_j> weighted by its C value, or
    // the change of an owned pair constraint
    auto apply_edge = [&](const T (&xj)[K][VEC], const T (&yj)[K][VEC], T cv, int cd) {
      T pd = (T)0;  // lane part of <D_i, Y_j> + <X_i, D_j>
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          pd = tfma(d[k][v], yj[k][v], pd);
          pd = tfma(x[k][v], yj[k][v] - xj[k][v], pd);
        }
      if (Tr::kDiag || cd == kNoCons) {
        cd_l = tfma(cv, pd, cd_l);
      } else {
        // owned pair constraint l: dT_l = <Y_i,Y_j> - <X_i,X_j>
        const T dt = group_sum<G>(pd, gmask);
        if (lane_g == 0) {
          const T rx = rXv[cd];
          acc_pd.add(pv[cd] * dt);
          acc_q.add(dt * ((T)2 * rx + dt));
          if (rYv) rYv[cd] = rx + dt;
        }
      }
    };
    // mirrored pair entries are done by the owner row; pure C entries only
    // in families with a sparse C
    auto skip = [&](int cd) {
      if (!Tr::kPairs) return false;
      return (cd < 0 && cd != kNoCons) || (!Tr::kCval && cd == kNoCons);
    };
    if constexpr (G == 1) {
      // one thread per row: entries two at a time, all gathers issued before
      // any is used
      int e = e0;
      for (; e + 2 <= e1; e += 2) {
        const int cd0 = Tr::kPairs ? a.code[e] : 0, cd1 = Tr::kPairs ? a.code[e + 1] : 0;
        const bool s0 = skip(cd0), s1 = skip(cd1);
        if (s0 && s1) continue;
        const int64_t j0 = a.col[e], j1 = a.col[e + 1];
        const T cv0 = Tr::kCval ? cval[e] : (T)0, cv1 = Tr::kCval ? cval[e + 1] : (T)0;
        T xj0[K][VEC], yj0[K][VEC], xj1[K][VEC], yj1[K][VEC];
        if (!s0) gather(j0, xj0, yj0);
        if (!s1) gather(j1, xj1, yj1);
        if (!s0) apply_edge(xj0, yj0, cv0, cd0);
        if (!s1) apply_edge(xj1, yj1, cv1, cd1);
      }
      if (e < e1) {
        const int cd0 = Tr::kPairs ? a.code[e] : 0;
        if (!skip(cd0)) {
          T xj0[K][VEC], yj0[K][VEC];
          gather(a.col[e], xj0, yj0);
          apply_edge(xj0, yj0, Tr::kCval ? cval[e] : (T)0, cd0);
        }
      }
    } else {
      // edge metadata in batches, as in k_grad
      for (int eb = e0; eb < e1; eb += kEdgeBatch<G>) {
        const int cnt = min(kEdgeBatch<G>, e1 - eb);
        int col_t = 0, code_t = 0;
        T cv_t = (T)0;
        if (lane_g < cnt) {
          col_t = a.col[eb + lane_g];
          if (Tr::kCval) cv_t = cval[eb + lane_g];
          if (Tr::kPairs) code_t = a.code[eb + lane_g];
        }
#pragma unroll
        for (int t = 0; t < kEdgeBatch<G>; ++t) {
          const T cv = Tr::kCval ? group_bcast<G>(cv_t, t, gmask) : (T)0;
          const int cd = Tr::kPairs ? group_bcast<G>(code_t, t, gmask) : 0;
          const int64_t j = group_bcast<G>(col_t, t, gmask);
          if (t >= cnt) continue;  // uniform over the group
          if (skip(cd)) continue;
          T xj[K][VEC], yj[K][VEC];
          gather(j, xj, yj);
          apply_edge(xj, yj, cv, cd);
        }
      }
    }
    acc_t0.add(cd_l + cdiag[i] * own_l);  // sparse C part and the diagonal of C
  }
  if constexpr (YZ) {
    Acc<T> red[8] = {acc_t0, acc_pd, acc_q, acc_tr, e0s, e1s, e2s, e3s};
    grid_reduce_acc<T, 8>(red, a.partials, a.counter, a.out);
  } else {
    Acc<T> red[4] = {acc_t0, acc_pd, acc_q, acc_tr};
    grid_reduce_acc<T, 4>(red, a.partials, a.counter, a.out);
  }
}

// ---------------------------------------------------------------------------
// pre-passes: column sums (C_J part) and |U|_F^2 (trace row)
// ---------------------------------------------------------------------------
// Thread t of a block owns column t mod ld of every (256 / ld)-th row; the
// per-thread sums are combined per column in a fixed order, so each block's
// partial row and the last block's total are deterministic.
// With cind (device memory, filled by the device-side ADAP-AIPP loop) U and Y
// come from there, an inactive cind makes the launch a no-op, and
// y_from_z reads Y as cs Z, cs = min(1, tau/sqrt(*z2)) (ADAP-FISTA's ball
// projection).
template <class T>
__global__ void __launch_bounds__(kBlock) k_colsum(const T* __restrict__ U, int64_t n, int ld,
                                                   int mode, const T* __restrict__ Y,
                                                   double* partials, unsigned* counter,
                                                   double* colsum_out, double* colsum_out2,
                                                   double* scal_out, double cj,
                                                   T* __restrict__ cj_out,
                                                   const ColInd* __restrict__ cind,
                                                   const double* __restrict__ z2, double tau) {
  // mode 0: s = colsum(U), scal = [|U|_F^2, |s|^2]
  // mode 1: X = U, D = Y - X: s = colsum(D), s2 = colsum(Y + X),
  //         scal = [sum <D_i, Y_i + X_i>, <s, s2>]
  __shared__ T s_ys;
  if (cind != nullptr) {
    const ColInd ci = *cind;
    if (!ci.active) return;  // uniform over the grid
    U = static_cast<const T*>(ci.U);
    Y = static_cast<const T*>(ci.Y);
    if (threadIdx.x == 0) {
      T v = (T)1;
      if (ci.y_from_z) {
        const double zn = sqrt(*z2);
        v = (T)(zn > tau ? tau / zn : 1.0);
      }
      s_ys = v;
    }
  } else if (threadIdx.x == 0) {
    s_ys = (T)1;
  }
  __syncthreads();
  const T ys = s_ys;
  __shared__ double t1[kBlock], t2[kBlock];
  __shared__ double sh[kColsumMax], sh2[kColsumMax];
  __shared__ double shr[1][kBlock / 32];
  __shared__ bool am_last;
  const int rows_per_pass = kBlock / ld > 0 ? kBlock / ld : 1;
  const int c = threadIdx.x % ld;
  const int rsub = threadIdx.x / ld;
  Acc<T> acc, acc2, nrm;
  if (rsub < rows_per_pass) {
    for (int64_t i = (int64_t)blockIdx.x * rows_per_pass + rsub; i < n;
         i += (int64_t)gridDim.x * rows_per_pass) {
      const T x = U[i * ld + c];
      if (mode == 0) {
        acc.add(x);
        nrm.add(x * x);
      } else {
        const T y = ys * Y[i * ld + c];
        const T dd = y - x;
        acc.add(dd);
        acc2.add(y + x);
        nrm.add(dd * (y + x));
      }
    }
  }
  t1[threadIdx.x] = acc.value();
  t2[threadIdx.x] = acc2.value();
  double red[1] = {nrm.value()};
  block_sum<1>(red, shr);  // contains __syncthreads
  const int W = ld + 1;
  for (int cc = threadIdx.x; cc < ld; cc += kBlock) {
    double s = 0.0, s2 = 0.0;
    for (int q = 0; q < rows_per_pass; ++q) {
      s += t1[q * ld + cc];
      s2 += t2[q * ld + cc];
    }
    partials[(size_t)blockIdx.x * (2 * W) + cc] = s;
    partials[(size_t)blockIdx.x * (2 * W) + W + cc] = s2;
  }
  if (threadIdx.x == 0) partials[(size_t)blockIdx.x * (2 * W) + ld] = red[0];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  for (int cc = threadIdx.x; cc <= ld; cc += kBlock) {
    double s = 0.0, s2 = 0.0;
    for (unsigned bb = 0; bb < gridDim.x; ++bb) {
      s += __ldcg(&partials[(size_t)bb * (2 * W) + cc]);
      if (cc < ld) s2 += __ldcg(&partials[(size_t)bb * (2 * W) + W + cc]);
    }
    if (cc < ld) {
      sh[cc] = s;
      sh2[cc] = s2;
      colsum_out[cc] = s;
      if (colsum_out2) colsum_out2[cc] = s2;
      if (cj_out) cj_out[cc] = (T)(cj * s);
    } else {
      scal_out[0] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int cc = 0; cc < ld; ++cc) q += (mode == 0 ? sh[cc] * sh[cc] : sh[cc] * sh2[cc]);
    scal_out[1] = q;
    *counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// r = A(YY^T) - b in double from the stored factor (thread per row, the
// owner entry of each pair constraint): the residuals of the dual update
// p <- p + beta r, the Lanczos shift p + beta r, the Frank-Wolfe step and the
// KKT primal residual.  In the mixed form the operator kernels' float
// residuals carry rounding of order 2^-24 |Y_i||Y_j|, which beta (up to 1e8)
// would amplify into the multipliers; here every product of the float
// factor is exact in double.  Reduces [sum r_l^2 (trace row excluded),
// |Y|_F^2]; the trace row's entry is left to the caller.
// ---------------------------------------------------------------------------
template <class T, int FAM>
__global__ void __launch_bounds__(kBlock) k_resid64(OpArgs a, const T* __restrict__ U, int r,
                                                    const double* __restrict__ bd,
                                                    double* __restrict__ r64) {
  using Tr = FamTraits<FAM>;
  double red[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kBlock) {
    const T* ui = U + i * (int64_t)a.ld;
    double nrm = 0.0;
    for (int k = 0; k < r; ++k) nrm = fma((double)ui[k], (double)ui[k], nrm);
    red[1] += nrm;
    if (Tr::kDiag) {
      const double rr = nrm - bd[i];
      r64[i] = rr;
      red[0] = fma(rr, rr, red[0]);
    } else {
      for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
        const int cd = a.code[e];
        if (cd < 0) continue;  // mirrored or pure C entry
        const T* uj = U + (int64_t)a.col[e] * a.ld;
        double dot = 0.0;
        for (int k = 0; k < r; ++k) dot = fma((double)ui[k], (double)uj[k], dot);
        const double rr = dot - bd[cd];
        r64[cd] = rr;
        red[0] = fma(rr, rr, red[0]);
      }
    }
  }
  grid_reduce<2>(red, a.partials, a.counter, a.out);
}

// ---------------------------------------------------------------------------
// Frank-Wolfe denominator sum_l (A_l.YY^T - tau^2 A_l.yy^T)^2 over the
// non-trace constraints, with A_l.YY^T = r_l + b_l (r = 1 gathers, FP64; run
// once per Frank-Wolfe step)
// ---------------------------------------------------------------------------
template <class T, int FAM>
__global__ void __launch_bounds__(kBlock) k_fw_denom(OpArgs a, const double* __restrict__ bd,
                                                     const double* __restrict__ y,
                                                     const T* __restrict__ resid, double tau2) {
  using Tr = FamTraits<FAM>;
  double red[2] = {0.0, 0.0};  // sum of squares, |y|^2
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kBlock) {
    const double yi = y[i];
    red[1] += yi * yi;
    if (Tr::kDiag) {
      const double dl = (double)resid[i] + bd[i] - tau2 * yi * yi;
      red[0] += dl * dl;
    } else {
      const int e0 = a.rowptr[i], e1 = a.rowptr[i + 1];
      for (int e = e0; e < e1; ++e) {
        const int cd = a.code[e];
        if (cd < 0) continue;  // mirrored or pure C entry
        const double dl = (double)resid[cd] + bd[cd] - tau2 * yi * __ldcg(&y[a.col[e]]);
        red[0] += dl * dl;
      }
    }
  }
  grid_reduce<2>(red, a.partials, a.counter, a.out);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
OpArgs make_args(Ctx* c, int ld, int slot) {
  const Problem& P = c->P;
  OpArgs a;
  a.n = P.n;
  a.ld = ld;
  a.rowptr = P.rowptr;
  a.col = P.col;
  a.code = P.code;
  const bool mixed = c->opt.precision == HALLAR_MIXED;
  a.cval = mixed ? (const void*)P.cval32 : (const void*)P.cval;
  a.cdiag = mixed ? (const void*)P.cdiag32 : (const void*)P.cdiag;
  a.b = mixed ? (const void*)P.b32 : (const void*)P.b;
  a.p = nullptr;
  a.C_J = P.C_J;
  a.beta = 0.0;
  a.has_trace = P.has_trace;
  a.trace_row = P.m - 1;
  a.partials = c->red.partials;
  a.counter = c->red.counter;
  a.out = c->d_scal + slot;
  return a;
}

struct Shape {
  int G, K;
};
Shape pick_shape(int ld, int vec) {
  const int nch = ld / vec;
  // narrow rows: one thread per row (K chunks each), so a warp keeps 32 rows'
  // gathers in flight and row sums need no shuffles; rows of 6-8 chunks: four
  // lanes of two chunks.  Measured on the 10^6-vertex torus: float r = 10
  // 44 us (88 us with four lanes of one chunk), float r = 32 111 us (152 us
  // with eight lanes of one chunk), double r = 10 158 us (453 us).
  if (nch <= 5) return {1, nch};
  if (nch <= 8) return {4, 2};
  if (nch <= 32) {
    int G = 8;
    while (G < nch) G <<= 1;
    return {G, 1};
  }
  const int K = (nch + 31) / 32;
  return {32, K <= 2 ? 2 : 4};
}

// run `body` with the row-group shape template arguments G and K for `ld`
#define HL_BY_SHAPE(T_, ld, ...)                                      \
  do {                                                                 \
    const Shape s__ = pick_shape((ld), V16<T_>::N);                    \
    switch (s__.G * 10 + s__.K) {                                      \
      case 11: { constexpr int G = 1, K = 1; __VA_ARGS__; } break;            \
      case 12: { constexpr int G = 1, K = 2; __VA_ARGS__; } break;            \
      case 13: { constexpr int G = 1, K = 3; __VA_ARGS__; } break;            \
      case 14: { constexpr int G = 1, K = 4; __VA_ARGS__; } break;            \
      case 15: { constexpr int G = 1, K = 5; __VA_ARGS__; } break;            \
      case 42: { constexpr int G = 4, K = 2; __VA_ARGS__; } break;            \
      case 81: { constexpr int G = 8, K = 1; __VA_ARGS__; } break;            \
      case 161: { constexpr int G = 16, K = 1; __VA_ARGS__; } break;          \
      case 321: { constexpr int G = 32, K = 1; __VA_ARGS__; } break;          \
      case 322: { constexpr int G = 32, K = 2; __VA_ARGS__; } break;          \
      case 324: { constexpr int G = 32, K = 4; __VA_ARGS__; } break;          \
      default: fail(HALLAR_EINVAL, "unsupported factor width");        \
    }                                                                  \
  } while (0)

// run `body` with T (factor type) and FAM (kernel family) of the handle
#define HL_BY_FAM_TYPE(c, ...)                                                         \
  do {                                                                                  \
    const bool mixed__ = (c)->opt.precision == HALLAR_MIXED;                            \
    switch ((c)->P.fam) {                                                               \
      case FAM_DIAG:                                                                    \
        if (mixed__) { using T = float; constexpr int FAM = FAM_DIAG; __VA_ARGS__; }           \
        else { using T = double; constexpr int FAM = FAM_DIAG; __VA_ARGS__; }                  \
        break;                                                                          \
      case FAM_EDGE:                                                                    \
        if (mixed__) { using T = float; constexpr int FAM = FAM_EDGE; __VA_ARGS__; }           \
        else { using T = double; constexpr int FAM = FAM_EDGE; __VA_ARGS__; }                  \
        break;                                                                          \
      default:                                                                          \
        if (mixed__) { using T = float; constexpr int FAM = FAM_EDGE_C; __VA_ARGS__; }         \
        else { using T = double; constexpr int FAM = FAM_EDGE_C; __VA_ARGS__; }                \
        break;                                                                          \
    }                                                                                   \
  } while (0)

}  // namespace

// Bytes of one operator launch: the factor rows (and W) once, the merged CSR
// once, the per-row and per-constraint vectors once; gathered neighbour rows
// are not counted.  alg counts the r columns of the factor and the element
// size the kernel reads per-row vectors in (4 bytes in the mixed form, 8 in
// FP64); pad counts the stored leading dimension ld instead of r.
OpBytes op_bytes(const Ctx* c, int r, int ld, int factor_arrays, bool writes_resid,
                 bool reads_p, bool reads_rx) {
  const Problem& P = c->P;
  const double es = (double)elem_size(c);
  double b = 0.0;
  b += (double)P.nnz * 4.0;                                      // column indices
  if (P.code) b += (double)P.nnz * 4.0;                          // constraint codes
  if (P.fam != FAM_EDGE) b += (double)P.nnz * es;                // C values
  b += (double)(P.n + 1) * 4.0 + (double)P.n * es;               // row pointers, diagonal
  const double mv = 1.0 + (reads_p ? 1.0 : 0.0) + (writes_resid ? 1.0 : 0.0) +
                    (reads_rx ? 1.0 : 0.0);
  b += (double)P.m * es * mv;                                    // b, p, r_X, r
  OpBytes o;
  o.alg = b + (double)P.n * r * es * factor_arrays;
  o.pad = b + (double)P.n * ld * es * factor_arrays;
  return o;
}

namespace {

template <int EPI>
void grad_dispatch(Ctx* c, const OpArgs& a, const GradIO& io, const GradInd& gi,
                   const GradInd* gind, int ld) {
  HL_BY_FAM_TYPE(c, HL_BY_SHAPE(T, ld, {
    if (io.cjv != nullptr) {
      const int grid = wave_grid(c, k_grad<T, FAM, G, K, true, EPI>, a.n, kBlock / G, kBlock);
      k_grad<T, FAM, G, K, true, EPI><<<grid, kBlock, 0, c->stream>>>(a, io, gi, gind);
    } else {
      const int grid = wave_grid(c, k_grad<T, FAM, G, K, false, EPI>, a.n, kBlock / G, kBlock);
      k_grad<T, FAM, G, K, false, EPI><<<grid, kBlock, 0, c->stream>>>(a, io, gi, gind);
    }
  }));
  HL_CHECK_LAUNCH(c);
}

template <bool YZ>
void change_dispatch(Ctx* c, const OpArgs& a, const DiffIO& io, const VcInd& vi,
                     const VcInd* vind, int ld) {
  HL_BY_FAM_TYPE(c, HL_BY_SHAPE(T, ld, {
    const int grid = wave_grid(c, k_value_change<T, FAM, G, K, YZ>, a.n, kBlock / G, kBlock);
    k_value_change<T, FAM, G, K, YZ><<<grid, kBlock, 0, c->stream>>>(a, io, vi, vind);
  }));
  HL_CHECK_LAUNCH(c);
}

}  // namespace

void launch_grad(Ctx* c, const void* U, int ld, int r, const void* p, double beta,
                 GradOut out) {
  if (ld > kColsumMax) fail(HALLAR_EINVAL, "factor width above 256");
  OpArgs a = make_args(c, ld, S_GRAD);
  a.p = p;
  const bool mixed = c->opt.precision == HALLAR_MIXED;
  GradIO io;
  io.cjv = (c->P.C_J != 0.0) ? cj_row(c) : nullptr;
  io.pre = c->d_scal + S_PRE;
  GradInd gi;
  gi.U = U;
  gi.out = out.W;
  gi.resid = out.resid;
  gi.beta = beta;
  gi.active = 1;
  // constraint values leave the kernel in the factor type (no double
  // instructions in the row loop); the float form widens them afterwards
  void* tout = nullptr;
  if (out.T)
    tout = mixed ? ensure_buffer(c, &c->stage_T, &c->stage_T_bytes, (size_t)c->P.m * sizeof(float))
                 : (void*)(out.T + 1);
  io.Tout = tout;
  const int tok = prof_begin(c, 0, op_bytes(c, r, ld, out.W != nullptr ? 2 : 1,
                                            out.resid != nullptr, true, false));
  grad_dispatch<EPI_W>(c, a, io, gi, nullptr, ld);
  prof_end(c, tok);
  if (out.T && mixed) launch_to_double(c, c->P.m, out.T + 1, tout);
}

void launch_grad_epi(Ctx* c, int epi, int ld, int r, const void* p, const GradInd* gind) {
  if (ld > kColsumMax) fail(HALLAR_EINVAL, "factor width above 256");
  OpArgs a = make_args(c, ld, S_GRAD);
  a.p = p;
  GradIO io;
  io.cjv = (c->P.C_J != 0.0) ? cj_row(c) : nullptr;
  io.pre = c->d_scal + S_PRE;
  io.Tout = nullptr;
  const GradInd unused;
  // factor arrays: x~, the centre and z out (FISTA); y, z and the centre (AIPP)
  const int tok = prof_begin(c, 0, op_bytes(c, r, ld, 3, true, true, false));
  if (epi == EPI_FISTA_Z) grad_dispatch<EPI_FISTA_Z>(c, a, io, unused, gind, ld);
  else grad_dispatch<EPI_AIPP>(c, a, io, unused, gind, ld);
  prof_end(c, tok);
}

void launch_value_change(Ctx* c, const void* X, const void* Y, int ld, int r, const void* p,
                         const void* rX, void* rY) {
  OpArgs a = make_args(c, ld, S_DIFF);
  a.p = p;
  DiffIO io{nullptr, 0.0};
  VcInd vi;
  vi.X = X;
  vi.Y = Y;
  vi.rX = rX;
  vi.rY = rY;
  vi.active = 1;
  const int tok = prof_begin(c, 1, op_bytes(c, r, ld, 2, rY != nullptr, true, true));
  change_dispatch<false>(c, a, io, vi, nullptr, ld);
  prof_end(c, tok);
}

void launch_value_change_ind(Ctx* c, bool y_from_z, int ld, int r, const void* p,
                             const VcInd* vind) {
  OpArgs a = make_args(c, ld, S_DIFF);
  a.p = p;
  DiffIO io{c->d_scal + S_GRAD + 4, std::sqrt(c->P.tau2)};
  const VcInd unused;
  if (y_from_z) {
    // x~, z and the centre in, y out
    const int tok = prof_begin(c, 1, op_bytes(c, r, ld, 4, false, true, true));
    change_dispatch<true>(c, a, io, unused, vind, ld);
    prof_end(c, tok);
  } else {
    const int tok = prof_begin(c, 1, op_bytes(c, r, ld, 2, false, true, true));
    change_dispatch<false>(c, a, io, unused, vind, ld);
    prof_end(c, tok);
  }
}

namespace {
template <class T>
void colsum_launch(Ctx* c, const void* U, int ld, int mode, const void* Y, double* out1,
                   double* out2, double* scal, void* cjo, const ColInd* cind) {
  const int rows_per_pass = kBlock / ld > 0 ? kBlock / ld : 1;
  const int grid = grid_for(c, c->P.n, rows_per_pass * 8);
  k_colsum<T><<<grid, kBlock, 0, c->stream>>>(
      (const T*)U, c->P.n, ld, mode, (const T*)Y, c->red.partials, c->red.counter, out1, out2,
      scal, mode == 0 ? c->P.C_J : 0.0, (T*)cjo, cind, c->d_scal + S_GRAD + 4,
      std::sqrt(c->P.tau2));
  HL_CHECK_LAUNCH(c);
}
}  // namespace

void launch_colsum(Ctx* c, const void* U, int ld, double* colsum_out, int slot) {
  if (ld > kColsumMax) fail(HALLAR_EINVAL, "factor width above 256");
  void* cjo = c->P.C_J != 0.0 ? cj_row(c) : nullptr;
  if (c->opt.precision == HALLAR_MIXED)
    colsum_launch<float>(c, U, ld, 0, nullptr, colsum_out, nullptr, c->d_scal + slot, cjo,
                         nullptr);
  else
    colsum_launch<double>(c, U, ld, 0, nullptr, colsum_out, nullptr, c->d_scal + slot, cjo,
                          nullptr);
}

void launch_colsum_ind(Ctx* c, int ld, const ColInd* cind) {
  if (ld > kColsumMax) fail(HALLAR_EINVAL, "factor width above 256");
  void* cjo = c->P.C_J != 0.0 ? cj_row(c) : nullptr;
  if (c->opt.precision == HALLAR_MIXED)
    colsum_launch<float>(c, nullptr, ld, 0, nullptr, c->d_colsum, nullptr, c->d_scal + S_PRE,
                         cjo, cind);
  else
    colsum_launch<double>(c, nullptr, ld, 0, nullptr, c->d_colsum, nullptr, c->d_scal + S_PRE,
                          cjo, cind);
}

void launch_colsum_diff(Ctx* c, const void* X, const void* Y, int ld, double* sD, double* sS) {
  if (ld > kColsumMax) fail(HALLAR_EINVAL, "factor width above 256");
  if (c->opt.precision == HALLAR_MIXED)
    colsum_launch<float>(c, X, ld, 1, Y, sD, sS, c->d_scal + S_DIFF + 8, nullptr, nullptr);
  else
    colsum_launch<double>(c, X, ld, 1, Y, sD, sS, c->d_scal + S_DIFF + 8, nullptr, nullptr);
}

void launch_colsum_diff_ind(Ctx* c, int ld, const ColInd* cind) {
  if (ld > kColsumMax) fail(HALLAR_EINVAL, "factor width above 256");
  double* sD = c->d_colsum + kColsumMax;
  double* sS = c->d_colsum + 2 * kColsumMax;
  if (c->opt.precision == HALLAR_MIXED)
    colsum_launch<float>(c, nullptr, ld, 1, nullptr, sD, sS, c->d_scal + S_DIFF + 8, nullptr,
                         cind);
  else
    colsum_launch<double>(c, nullptr, ld, 1, nullptr, sD, sS, c->d_scal + S_DIFF + 8, nullptr,
                          cind);
}

void launch_fw_denom(Ctx* c, const double* y, const double* resid, double tau2, int slot) {
  OpArgs a = make_args(c, 1, slot);
  const int grid = grid_for(c, c->P.n, kBlock);
  switch (c->P.fam) {
    case FAM_DIAG:
      k_fw_denom<double, FAM_DIAG><<<grid, kBlock, 0, c->stream>>>(a, c->P.b, y, resid, tau2);
      break;
    case FAM_EDGE:
      k_fw_denom<double, FAM_EDGE><<<grid, kBlock, 0, c->stream>>>(a, c->P.b, y, resid, tau2);
      break;
    default:
      k_fw_denom<double, FAM_EDGE_C><<<grid, kBlock, 0, c->stream>>>(a, c->P.b, y, resid, tau2);
      break;
  }
  HL_CHECK_LAUNCH(c);
}

void launch_resid64(Ctx* c, const void* U, int ld, int r, double* r64, int slot) {
  OpArgs a = make_args(c, ld, slot);
  const int grid = grid_for(c, c->P.n, kBlock);
  HL_BY_FAM_TYPE(c, {
    k_resid64<T, FAM><<<grid, kBlock, 0, c->stream>>>(a, (const T*)U, r, c->P.b, r64);
  });
  HL_CHECK_LAUNCH(c);
}

}  // namespace hallar
