// Minimum eigenpair of G = C + A*(p') (Alg. 1 step 7, eq. Grad X Space) by
// Lanczos with partial reorthogonalisation, in FP64 for both precision forms.
//
// A plain step is two thread-per-row passes over n-vectors:
//   step 1  w = G q_k - beta_{k-1} q_{k-1}, alpha_k = <q_k, w>, q_k -> Q[:, k]
//   step 2  w <- w - alpha_k q_k (alpha_k read from device memory),
//           |w|^2 and sum(w)
// and one host sync.  The host tracks the loss of orthogonality with
// Simon's recurrence for omega_{k+1,j} ~ q_{k+1}^T q_j (H. D. Simon, "The
// Lanczos algorithm with partial reorthogonalization", Math. Comp. 42, 1984);
// when an estimate passes sqrt(eps), w is orthogonalised against the whole
// basis by two classical Gram-Schmidt sweeps, at that step and the next.
// Semi-orthogonality keeps the Ritz values of the tridiagonal accurate to
// O(eps |G|), as full reorthogonalisation does, at a fraction of the FP64
// work (a sweep costs two FMAs per basis element on the slow FP64 pipe).
//
// The basis Q is stored row-major, n x kcap (row i holds q_0[i] .. q_k[i]),
// so a sweep streams Q with coalesced row reads, one warp per row:
//   sweep a  h = Q^T w                     (k_lan_orth with h = 0)
//   sweep b  w <- w - Q h and h2 = Q^T w   (k_lan_orth)
//   sweep c  w <- w - Q h2, |w|^2, sum(w)  (k_lan_final)
// The host solves the k x k tridiagonal (Sturm bisection + inverse
// iteration) and tests the Ritz residual.
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

namespace {

constexpr int kLanMaxCols = 512;  // 16 accumulators per lane

// Lanczos vectors are unpadded FP64 n-vectors: algorithmic = stored bytes
OpBytes lan_bytes(double b) {
  OpBytes o;
  o.alg = o.pad = b;
  return o;
}

struct LanArgs {
  int64_t n;
  const int* __restrict__ rowptr;
  const int* __restrict__ col;
  const int* __restrict__ code;
  const double* __restrict__ cval;
  const double* __restrict__ cdiag;
  double C_J;
  int fam;
  int has_trace;
  int64_t trace_row;
  const double* __restrict__ ps;  // p'
};

// per-warp partial column sums -> per-block partial rows (fixed order)
template <int NACC>
__device__ inline void write_block_partial(double (&acc)[NACC], int ncols,
                                           double* __restrict__ part) {
  __shared__ double sh[kBlock / 32][kLanMaxCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NACC; ++t) {
    const int j = lane + 32 * t;
    if (j < ncols) sh[warp][j] = acc[t];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ncols; j += kBlock) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += sh[w][j];
    part[(size_t)blockIdx.x * ncols + j] = s;
  }
}

__device__ inline double gv_row(const LanArgs& a, int64_t i, const double* __restrict__ v,
                                 double vscale, double vsum, double vi, int lane, int stride) {
  // lanes lane, lane + stride, ... of the row's entries; caller reduces
  double s = 0.0;
  for (int e = a.rowptr[i] + lane; e < a.rowptr[i + 1]; e += stride) {
    const double vj = __ldcg(&v[a.col[e]]) * vscale;
    double coef;
    if (a.fam == FAM_DIAG) {
      coef = a.cval[e];
    } else {
      const int cd = a.code[e];
      coef = cd == kNoCons ? a.cval[e] : 0.5 * a.ps[cd >= 0 ? cd : -cd - 1];
    }
    s = fma(coef, vj, s);
  }
  if (lane == 0) {
    double dc = a.cdiag[i];
    if (a.fam == FAM_DIAG) dc += a.ps[i];
    else if (a.has_trace) dc += a.ps[a.trace_row];
    s = fma(dc, vi, s) + a.C_J * vsum;
  }
  return s;
}

// step 1: q_k = vin * vscale (stored as column k of Q),
// w = G q_k - bprev * (prev * pscale) written over prev, alpha partial <q_k, w>
__global__ void __launch_bounds__(kBlock) k_lan_step1(LanArgs a, const double* __restrict__ vin,
                                                      double vscale, double vsum,
                                                      double* __restrict__ prev, double pscale,
                                                      double bprev, double* __restrict__ Q,
                                                      int kcap, int k, double* partials,
                                                      unsigned* counter, double* out) {
  double red[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kBlock) {
    const double vi = vin[i] * vscale;
    double wi = gv_row(a, i, vin, vscale, vsum, vi, 0, 1);
    if (bprev != 0.0) wi = fma(-bprev * pscale, prev[i], wi);
    prev[i] = wi;
    Q[i * (int64_t)kcap + k] = vi;
    red[0] = fma(vi, wi, red[0]);
  }
  grid_reduce<1>(red, partials, counter, out);
}

// step 2: w <- w - alpha q_k, alpha = *alpha_dev; |w|^2 and sum(w)
__global__ void __launch_bounds__(kBlock) k_lan_step2(int64_t n, const double* __restrict__ vin,
                                                      double vscale,
                                                      const double* __restrict__ alpha_dev,
                                                      double* __restrict__ w, double* partials,
                                                      unsigned* counter, double* out) {
  const double am = -(*alpha_dev) * vscale;
  double red[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock) {
    const double wi = fma(am, vin[i], w[i]);
    w[i] = wi;
    red[0] = fma(wi, wi, red[0]);
    red[1] += wi;
  }
  grid_reduce<2>(red, partials, counter, out);
}

// sweep: w <- w - Q h and h2 = Q^T w   (ncols = k + 1; h = 0 gives h2 = Q^T w)
template <int NACC>
__global__ void __launch_bounds__(kBlock) k_lan_orth(int64_t n, const double* __restrict__ Q,
                                                     int kcap, int ncols,
                                                     const double* __restrict__ h,
                                                     double* __restrict__ w,
                                                     double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (kBlock / 32);
  double hv[NACC], acc[NACC];
#pragma unroll
  for (int t = 0; t < NACC; ++t) {
    const int j = lane + 32 * t;
    hv[t] = j < ncols ? h[j] : 0.0;
    acc[t] = 0.0;
  }
  for (int64_t i = warp; i < n; i += nwarps) {
    const double* __restrict__ qrow = Q + i * (int64_t)kcap;
    double q[NACC];
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < NACC; ++t) {
      const int j = lane + 32 * t;
      q[t] = j < ncols ? qrow[j] : 0.0;
      s = fma(q[t], hv[t], s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const double wi = w[i] - s;
#pragma unroll
    for (int t = 0; t < NACC; ++t) acc[t] = fma(q[t], wi, acc[t]);
    __syncwarp();
    if (lane == 0) w[i] = wi;
  }
  write_block_partial<NACC>(acc, ncols, part);
}

// last sweep: w <- w - Q h2; reductions |w|^2 and sum(w) (ncols = 0: only the sums)
template <int NACC>
__global__ void __launch_bounds__(kBlock) k_lan_final(int64_t n, const double* __restrict__ Q,
                                                      int kcap, int ncols,
                                                      const double* __restrict__ h,
                                                      double* __restrict__ w, double* partials,
                                                      unsigned* counter, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (kBlock / 32);
  double hv[NACC];
#pragma unroll
  for (int t = 0; t < NACC; ++t) {
    const int j = lane + 32 * t;
    hv[t] = j < ncols ? h[j] : 0.0;
  }
  double red[2] = {0.0, 0.0};
  for (int64_t i = warp; i < n; i += nwarps) {
    const double* __restrict__ qrow = Q + i * (int64_t)kcap;
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < NACC; ++t) {
      const int j = lane + 32 * t;
      if (j < ncols) s = fma(qrow[j], hv[t], s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const double wi = w[i] - s;
    __syncwarp();
    if (lane == 0) {
      if (ncols > 0) w[i] = wi;
      red[0] += wi * wi;
      red[1] += wi;
    }
  }
  grid_reduce<2>(red, partials, counter, out);
}

// v = Q s (Ritz vector), |v|^2 into out[0]
template <int NACC>
__global__ void __launch_bounds__(kBlock) k_lan_combine(int64_t n, const double* __restrict__ Q,
                                                        int kcap, int ncols,
                                                        const double* __restrict__ s,
                                                        double* __restrict__ v, double* partials,
                                                        unsigned* counter, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (kBlock / 32);
  double sv[NACC];
#pragma unroll
  for (int t = 0; t < NACC; ++t) {
    const int j = lane + 32 * t;
    sv[t] = j < ncols ? s[j] : 0.0;
  }
  double red[1] = {0.0};
  for (int64_t i = warp; i < n; i += nwarps) {
    const double* __restrict__ qrow = Q + i * (int64_t)kcap;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < NACC; ++t) {
      const int j = lane + 32 * t;
      if (j < ncols) acc = fma(qrow[j], sv[t], acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      v[i] = acc;
      red[0] += acc * acc;
    }
  }
  grid_reduce<1>(red, partials, counter, out);
}

// sum the per-block partial rows: out[j] = sum_b part[b][j], one warp per column
__global__ void k_sum_cols(const double* __restrict__ part, int nblocks, int ncols,
                           double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ncols) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += part[(size_t)b * ncols + j];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) out[j] = s;
}

// SplitMix64 (Steele, Lea and Flood 2014): element k (1-based) of stream
// `seed` is the 64-bit finaliser of seed + k * 0x9E3779B97F4A7C15; the top
// 53 bits give u in [0, 1) and the value used is 2u - 1.
__global__ void k_splitmix(uint64_t seed, int64_t n, double* __restrict__ out, double mix_scale,
                           const double* __restrict__ base) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    const double r = 2.0 * u - 1.0;
    out[i] = base ? base[i] + mix_scale * r : r;
  }
}

__global__ void k_dscale(int64_t n, double* __restrict__ v, double s) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock)
    v[i] *= s;
}

// |G v - lambda v|^2 (one thread per row)
__global__ void __launch_bounds__(kBlock) k_lan_resid(LanArgs a, const double* __restrict__ v,
                                                      double vsum, double lambda,
                                                      double* partials, unsigned* counter,
                                                      double* out) {
  double red[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * kBlock) {
    const double gv = gv_row(a, i, v, 1.0, vsum, v[i], 0, 1);
    const double d = gv - lambda * v[i];
    red[0] += d * d;
  }
  grid_reduce<1>(red, partials, counter, out);
}

// ---------------------------------------------------------------------------
// host: smallest eigenpair of a symmetric tridiagonal matrix
// ---------------------------------------------------------------------------
// Sturm count: number of eigenvalues below x of T = tridiag(beta, alpha, beta),
// from the signs of the pivots of T - x I = L D L^T.
int sturm_count(const std::vector<double>& al, const std::vector<double>& be, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
    d = (al[i] - x) - (i > 0 ? b2 / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// smallest eigenvalue by bisection on the Sturm count, eigenvector by
// inverse iteration with a shift just below it
double tridiag_min_eig(const std::vector<double>& al, const std::vector<double>& be, int k,
                       std::vector<double>& s) {
  double lo = al[0], hi = al[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(be[i]) : 0.0);
    lo = std::fmin(lo, al[i] - r);
    hi = std::fmax(hi, al[i] + r);
  }
  const double scale = std::fmax(std::fabs(lo), std::fabs(hi));
  for (int it = 0; it < 200 && hi - lo > 4e-16 * scale; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(al, be, k, mid) >= 1) hi = mid;
    else lo = mid;
  }
  const double lam = 0.5 * (lo + hi);
  const double sigma = lam - 1e-13 * std::fmax(1.0, scale);
  s.assign(k, 1.0);
  std::vector<double> dd(k), x(k);
  for (int rep = 0; rep < 3; ++rep) {
    // (T - sigma I) x = s by Gaussian elimination without pivoting: T - sigma I
    // is positive definite up to rounding since sigma is below lambda_min
    double piv = al[0] - sigma;
    if (std::fabs(piv) < 1e-300) piv = 1e-300;
    dd[0] = piv;
    x[0] = s[0];
    for (int i = 1; i < k; ++i) {
      const double l = be[i - 1] / dd[i - 1];
      double p = (al[i] - sigma) - l * be[i - 1];
      if (std::fabs(p) < 1e-300) p = 1e-300;
      dd[i] = p;
      x[i] = s[i] - l * x[i - 1];
    }
    x[k - 1] /= dd[k - 1];
    for (int i = k - 2; i >= 0; --i) x[i] = (x[i] - be[i] * x[i + 1]) / dd[i];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += x[i] * x[i];
    nrm = std::sqrt(nrm);
    for (int i = 0; i < k; ++i) s[i] = x[i] / nrm;
  }
  return lam;
}

// run `body` with NACC = accumulators per lane for `ncols` basis columns
#define HL_BY_NACC(ncols, ...)                        \
  do {                                                \
    if ((ncols) <= 32) {                              \
      constexpr int NACC = 1;                         \
      __VA_ARGS__;                                    \
    } else if ((ncols) <= 64) {                       \
      constexpr int NACC = 2;                         \
      __VA_ARGS__;                                    \
    } else if ((ncols) <= 128) {                      \
      constexpr int NACC = 4;                         \
      __VA_ARGS__;                                    \
    } else if ((ncols) <= 256) {                      \
      constexpr int NACC = 8;                         \
      __VA_ARGS__;                                    \
    } else {                                          \
      constexpr int NACC = 16;                        \
      __VA_ARGS__;                                    \
    }                                                 \
  } while (0)

}  // namespace

void launch_splitmix(Ctx* c, uint64_t seed, double* out, double mix_scale, const double* base) {
  k_splitmix<<<grid_for(c, c->P.n, kBlock * 4), kBlock, 0, c->stream>>>(seed, c->P.n, out,
                                                                        mix_scale, base);
  HL_CHECK_LAUNCH(c);
}

LanczosOut lanczos_min_eig(Ctx* c, const double* pshift, const double* v0, double tol, int kmax,
                           int max_restarts, double* v_out) {
  const int64_t n = c->P.n;
  if (kmax < 2) kmax = 2;
  if (kmax > kLanMaxCols) kmax = kLanMaxCols;
  if (kmax > n) kmax = (int)n;
  const int kcap = (kmax + 3) / 4 * 4;
  int grid = grid_for(c, n, (kBlock / 32) * 4);
  if (grid > 1184) grid = 1184;
  const int grid_row = grid_for(c, n, kBlock * 2);
  // workspace kept by the handle between calls
  double* Q = (double*)ensure_buffer(c, &c->lan_Q, &c->lan_Q_bytes,
                                     (size_t)n * kcap * sizeof(double));
  double* bufs = (double*)ensure_buffer(c, &c->lan_w, &c->lan_w_bytes,
                                        2 * (size_t)n * sizeof(double));
  double* part = (double*)ensure_buffer(c, &c->lan_part, &c->lan_part_bytes,
                                        (size_t)grid * kcap * sizeof(double));
  double* hbuf = (double*)ensure_buffer(c, &c->lan_h, &c->lan_h_bytes,
                                        3 * (size_t)kcap * sizeof(double));
  double* h = hbuf;
  double* h2 = hbuf + kcap;
  double* sdev = hbuf + 2 * kcap;
  LanArgs a;
  a.n = n;
  a.rowptr = c->P.rowptr;
  a.col = c->P.col;
  a.code = c->P.code;
  a.cval = c->P.cval;
  a.cdiag = c->P.cdiag;
  a.C_J = c->P.C_J;
  a.fam = c->P.fam;
  a.has_trace = c->P.has_trace;
  a.trace_row = c->P.m - 1;
  a.ps = pshift;
  double* const d_alpha = c->d_scal + S_LAN + 6;  // alpha_k of the current step
  const double eps = 1.1102230246251565e-16;      // 2^-53
  const double sqrt_eps = std::sqrt(eps);
  const double omega_floor = eps * std::sqrt((double)n);  // omega after a sweep

  // |v|^2 and sum(v) of a vector: the last sweep with no basis columns
  auto norm_and_sum = [&](double* vec, double& nrm2, double& sum) {
    k_lan_final<1><<<grid, kBlock, 0, c->stream>>>(n, Q, kcap, 0, h, vec, c->red.partials,
                                                   c->red.counter, c->d_scal + S_LAN + 4);
    HL_CHECK_LAUNCH(c);
    fetch_scalars(c, S_LAN + 4, 2);
    nrm2 = c->h_scal[S_LAN + 4];
    sum = c->h_scal[S_LAN + 5];
  };

  double* vin = bufs + n;  // current basis vector, unnormalised
  double* prev = bufs;     // previous basis vector, then w
  HL_CUDA(cudaMemcpyAsync(vin, v0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  LanczosOut res{0.0, INFINITY, 0, false, 0};
  std::vector<double> al, be, s;
  std::vector<double> om_prev, om_cur, om_next;  // omega_{k-1,.}, omega_{k,.}, omega_{k+1,.}
  int total = 0;
  for (int restart = 0; restart <= max_restarts; ++restart) {
    double nv2, vs;
    norm_and_sum(vin, nv2, vs);
    if (!(nv2 > 0.0) || !std::isfinite(nv2)) {
      // degenerate start vector: use the SplitMix64 vector of the seed
      launch_splitmix(c, c->opt.seed + 1, vin, 0.0, nullptr);
      norm_and_sum(vin, nv2, vs);
    }
    double vscale = 1.0 / std::sqrt(nv2);
    double vsum = vs * vscale;
    double pscale = 0.0, bprev = 0.0;
    al.clear();
    be.clear();
    om_prev.assign(kmax + 2, 0.0);
    om_cur.assign(kmax + 2, 0.0);
    om_next.assign(kmax + 2, 0.0);
    om_cur[0] = 1.0;  // omega_{0,0}
    double anorm = 0.0;
    bool force_sweep = false;
    bool done = false;
    int kk = 0;
    for (int k = 0; k < kmax; ++k) {
      const int ncols = k + 1;
      // step 1 and step 2 (three-term recurrence)
      const int tok1 = prof_begin(c, 2, lan_bytes(40.0 * n + 12.0 * (double)c->P.nnz + 8.0 * c->P.m));
      k_lan_step1<<<grid_row, kBlock, 0, c->stream>>>(a, vin, vscale, vsum, prev, pscale, bprev, Q,
                                                     kcap, k, c->red.partials, c->red.counter,
                                                     d_alpha);
      HL_CHECK_LAUNCH(c);
      k_lan_step2<<<grid_row, kBlock, 0, c->stream>>>(n, vin, vscale, d_alpha, prev,
                                                     c->red.partials, c->red.counter,
                                                     c->d_scal + S_LAN);
      HL_CHECK_LAUNCH(c);
      prof_end(c, tok1);
      fetch_scalars(c, S_LAN, 7);
      ++total;
      double alpha = c->h_scal[S_LAN + 6];
      double bnorm = std::sqrt(c->h_scal[S_LAN]);
      double wsum = c->h_scal[S_LAN + 1];
      if (!std::isfinite(alpha) || !std::isfinite(bnorm))
        fail(HALLAR_ENUMERIC, "Lanczos: non-finite value");
      anorm = std::fmax(anorm, std::fabs(alpha) + bnorm + (k > 0 ? be[k - 1] : 0.0));

      // Simon's estimate of omega_{k+1,j} = q_{k+1}^T q_j, j <= k
      const bool forced = force_sweep;
      bool sweep = forced;
      if (bnorm > 0.0) {
        const double theta = 2.0 * eps * anorm / bnorm;
        for (int j = 0; j < k; ++j) {
          double o = be[j] * om_cur[j + 1] + (al[j] - alpha) * om_cur[j] - be[k - 1] * om_prev[j];
          if (j > 0) o += be[j - 1] * om_cur[j - 1];
          o /= bnorm;
          o += o >= 0.0 ? theta : -theta;
          om_next[j] = o;
          if (std::fabs(o) > sqrt_eps) sweep = true;
        }
        om_next[k] = eps * std::sqrt((double)n) * anorm / bnorm;
        if (std::fabs(om_next[k]) > sqrt_eps) sweep = true;
      }
      if (sweep && bnorm > 0.0) {
        // two classical Gram-Schmidt sweeps of w against q_0 .. q_k
        const int tok2 = prof_begin(c, 2, lan_bytes(3.0 * (8.0 * n * ncols + 16.0 * n)));
        HL_CUDA(cudaMemsetAsync(h2, 0, ncols * sizeof(double), c->stream));
        HL_BY_NACC(ncols, k_lan_orth<NACC><<<grid, kBlock, 0, c->stream>>>(n, Q, kcap, ncols, h2,
                                                                            prev, part));
        HL_CHECK_LAUNCH(c);
        k_sum_cols<<<(ncols * 32 + 255) / 256, 256, 0, c->stream>>>(part, grid, ncols, h);
        HL_CHECK_LAUNCH(c);
        HL_BY_NACC(ncols, k_lan_orth<NACC><<<grid, kBlock, 0, c->stream>>>(n, Q, kcap, ncols, h,
                                                                            prev, part));
        HL_CHECK_LAUNCH(c);
        k_sum_cols<<<(ncols * 32 + 255) / 256, 256, 0, c->stream>>>(part, grid, ncols, h2);
        HL_CHECK_LAUNCH(c);
        HL_BY_NACC(ncols, k_lan_final<NACC><<<grid, kBlock, 0, c->stream>>>(
                              n, Q, kcap, ncols, h2, prev, c->red.partials, c->red.counter,
                              c->d_scal + S_LAN));
        HL_CHECK_LAUNCH(c);
        prof_end(c, tok2);
        HL_CUDA(cudaMemcpyAsync(c->h_scal + S_LAN + 2, h + k, sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
        HL_CUDA(cudaMemcpyAsync(c->h_scal + S_LAN + 3, h2 + k, sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
        fetch_scalars(c, S_LAN, 2);
        // the components removed along q_k belong to alpha_k
        alpha += c->h_scal[S_LAN + 2] + c->h_scal[S_LAN + 3];
        bnorm = std::sqrt(c->h_scal[S_LAN]);
        wsum = c->h_scal[S_LAN + 1];
        if (!std::isfinite(alpha) || !std::isfinite(bnorm))
          fail(HALLAR_ENUMERIC, "Lanczos: non-finite value");
        for (int j = 0; j <= k; ++j) om_next[j] = omega_floor;
        // Simon: a sweep at one step is followed by a sweep at the next
        force_sweep = !forced;
        ++res.sweeps;
      } else {
        force_sweep = false;
      }
      om_next[k + 1] = 1.0;
      al.push_back(alpha);
      be.push_back(bnorm);
      kk = k + 1;
      res.lambda = tridiag_min_eig(al, be, kk, s);
      res.resid = std::fabs(bnorm * s[kk - 1]);
      if (res.resid <= tol || bnorm <= 1e-300 || kk == n) {
        done = true;
        break;
      }
      // next basis vector w / |w|, scaled on the fly by the next step 1
      std::swap(om_prev, om_cur);
      std::swap(om_cur, om_next);
      pscale = vscale;
      bprev = bnorm;
      vscale = 1.0 / bnorm;
      vsum = wsum * vscale;
      std::swap(vin, prev);
    }
    // Ritz vector v = Q s, normalised
    HL_CUDA(cudaMemcpyAsync(sdev, s.data(), kk * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream));
    HL_BY_NACC(kk, k_lan_combine<NACC><<<grid, kBlock, 0, c->stream>>>(
                       n, Q, kcap, kk, sdev, v_out, c->red.partials, c->red.counter,
                       c->d_scal + S_LAN));
    HL_CHECK_LAUNCH(c);
    fetch_scalars(c, S_LAN, 1);
    k_dscale<<<grid_for(c, n, kBlock * 4), kBlock, 0, c->stream>>>(
        n, v_out, 1.0 / std::sqrt(c->h_scal[S_LAN]));
    HL_CHECK_LAUNCH(c);
    // true residual |G v - lambda v| of the Ritz pair
    double vn2, vsv;
    norm_and_sum(v_out, vn2, vsv);
    k_lan_resid<<<grid_for(c, n, kBlock * 4), kBlock, 0, c->stream>>>(
        a, v_out, vsv, res.lambda, c->red.partials, c->red.counter, c->d_scal + S_LAN);
    HL_CHECK_LAUNCH(c);
    fetch_scalars(c, S_LAN, 1);
    res.resid = std::sqrt(c->h_scal[S_LAN]);
    res.iters = total;
    if (done && (res.resid <= 1.5 * tol || kk == n)) {
      res.converged = res.resid <= 1.5 * tol;
      break;
    }
    // restart from the Ritz vector
    HL_CUDA(cudaMemcpyAsync(vin, v_out, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  return res;
}

}  // namespace hallar
