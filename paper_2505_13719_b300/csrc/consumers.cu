// Consumers of a solved factor U (not in the paper, which stops at the SDP
// solution; they turn X = UU^T into the answers its applications want):
//
// * Goemans-Williamson hyperplane rounding for Max-Cut: for a hyperplane
//   normal g, x_i = sign(<U_i, g>) (+1 at 0), and the cut value of x is
//   -x^T C x (C = -L/4 for the Max-Cut SDP, so -x^T C x = (1/4) x^T L x =
//   the weight of the edges x cuts).  The caller passes the normals, so a
//   run is reproducible and the oracle can round with the same ones.
// * Entries of X = UU^T at given index pairs, X_ab = <U_a, U_b>: for a
//   matrix-completion problem (eq. matcomp-sdp) the recovered matrix is the
//   off-diagonal block, M^_ij = X_{i, n1 + j}.
//
// Both are gathers over U with FP64 arithmetic (the sign decisions and the
// cut sums are taken in double from the stored factor).
#include <cmath>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

namespace {

// x_i = sign(<U_i, g>) in double, +1 at zero
template <class T>
__global__ void __launch_bounds__(kBlock) k_round_sign(const T* __restrict__ U, int64_t n, int ld,
                                                       int r, const double* __restrict__ g,
                                                       int8_t* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock) {
    double s = 0.0;
    for (int k = 0; k < r; ++k) s = fma((double)U[i * ld + k], g[k], s);
    x[i] = s < 0.0 ? (int8_t)-1 : (int8_t)1;
  }
}

// x^T C x over the stored off-diagonal entries and the diagonal (C_I
// included), and sum x (for the C_J 11^T part): out[0], out[1]
__global__ void __launch_bounds__(kBlock) k_cut(int64_t n, const int* __restrict__ rowptr,
                                                const int* __restrict__ col,
                                                const double* __restrict__ cval,
                                                const double* __restrict__ cdiag,
                                                const int8_t* __restrict__ x, double* partials,
                                                unsigned* counter, double* out) {
  double red[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock) {
    const double xi = (double)x[i];
    double s = cdiag[i] * xi;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s = fma(cval[e], (double)x[col[e]], s);
    red[0] = fma(xi, s, red[0]);
    red[1] += xi;
  }
  grid_reduce<2>(red, partials, counter, out);
}

// X_ab = <U_a, U_b> for listed pairs, in double
template <class T>
__global__ void __launch_bounds__(kBlock) k_entries(const T* __restrict__ U, int ld, int r,
                                                    const int32_t* __restrict__ a,
                                                    const int32_t* __restrict__ b, int64_t count,
                                                    double* __restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * kBlock + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * kBlock) {
    const int64_t ia = a[t], ib = b[t];
    double s = 0.0;
    for (int k = 0; k < r; ++k) s = fma((double)U[ia * ld + k], (double)U[ib * ld + k], s);
    out[t] = s;
  }
}

}  // namespace

void launch_round_sign(Ctx* c, const void* U, int ld, int r, const double* g, int8_t* x) {
  const int grid = grid_for(c, c->P.n, kBlock);
  if (c->opt.precision == HALLAR_MIXED)
    k_round_sign<float><<<grid, kBlock, 0, c->stream>>>((const float*)U, c->P.n, ld, r, g, x);
  else
    k_round_sign<double><<<grid, kBlock, 0, c->stream>>>((const double*)U, c->P.n, ld, r, g, x);
  HL_CHECK_LAUNCH(c);
}

void launch_cut(Ctx* c, const int8_t* x, int slot) {
  const Problem& P = c->P;
  const int grid = grid_for(c, P.n, kBlock);
  k_cut<<<grid, kBlock, 0, c->stream>>>(P.n, P.rowptr, P.col, P.cval, P.cdiag, x,
                                        c->red.partials, c->red.counter, c->d_scal + slot);
  HL_CHECK_LAUNCH(c);
}

void launch_entries(Ctx* c, const void* U, int ld, int r, const int32_t* a, const int32_t* b,
                    int64_t count, double* out) {
  const int grid = grid_for(c, count, kBlock);
  if (c->opt.precision == HALLAR_MIXED)
    k_entries<float><<<grid, kBlock, 0, c->stream>>>((const float*)U, ld, r, a, b, count, out);
  else
    k_entries<double><<<grid, kBlock, 0, c->stream>>>((const double*)U, ld, r, a, b, count, out);
  HL_CHECK_LAUNCH(c);
}

}  // namespace hallar
