// Streaming kernels: the start factor's ball projection, the Frank-Wolfe
// rank update (eq. tilde Y), the rank trim and the m-vector operations of
// the dual update.  Every factor kernel is one pass over n x ld arrays with
// 16-byte vector accesses and folds the norms the host needs into the same
// pass (deterministic grid reduction).  Padding columns are zero and every
// update here is linear, so they stay zero.  (The ADAP-FISTA / ADAP-AIPP
// vector steps are fused into the operator kernels, and the x / x~ updates
// run in loop.cu.)
#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

namespace {

template <class T, int NS, class Op>
__global__ void __launch_bounds__(kBlock) k_stream(int64_t nvec, Op op, double* partials,
                                                   unsigned* counter, double* out) {
  Acc<T> red[NS > 0 ? NS : 1];
  Op o = op;
  o.setup();  // per-thread constants, computed once
  for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < nvec;
       v += (int64_t)gridDim.x * kBlock)
    o(v, red);
  if constexpr (NS > 0) grid_reduce_acc<T, NS>(red, partials, counter, out);
}

template <class T, int NS, class Op>
void run_stream(Ctx* c, int64_t nelem, const Op& op, int slot) {
  constexpr int VEC = V16<T>::N;
  const int64_t nvec = nelem / VEC;
  const int grid = wave_grid(c, k_stream<T, NS, Op>, nvec, kBlock * 4, kBlock);
  k_stream<T, NS, Op><<<grid, kBlock, 0, c->stream>>>(nvec, op, c->red.partials, c->red.counter,
                                                      c->d_scal + (slot >= 0 ? slot : 0));
  HL_CHECK_LAUNCH(c);
}

#define HL_LOAD(ptr, v, arr) load_chunk<T>((ptr), (v) * VEC, arr)

// every element operation runs in the factor type T (float in the mixed
// form: double instructions are the scarce resource on B300); reductions
// accumulate in Acc<T>
struct OpBase {
  __device__ void setup() {}
};

template <class T>
struct OpScale : OpBase {
  T* u; T s;
  __device__ void operator()(int64_t v, Acc<T>*) const {
    constexpr int VEC = V16<T>::N;
    T a[VEC];
    HL_LOAD(u, v, a);
#pragma unroll
    for (int k = 0; k < VEC; ++k) a[k] = s * a[k];
    store_chunk<T>(u, v * VEC, a);
  }
};

template <class T>
struct OpNorm2 : OpBase {
  const T* u;
  __device__ void operator()(int64_t v, Acc<T>* red) const {
    constexpr int VEC = V16<T>::N;
    T a[VEC];
    HL_LOAD(u, v, a);
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < VEC; ++k) s = tfma(a[k], a[k], s);
    red[0].add(s);
  }
};

// padded, scaled row copy: dst[i, 0:r_copy] = s * src[i, 0:r_copy], rest 0
template <class T>
__global__ void k_pad_copy(const T* __restrict__ src, int ld_src, T* __restrict__ dst, int ld_dst,
                           int r_copy, int64_t n, T s) {
  const int64_t total = n * ld_dst;
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kBlock) {
    const int64_t i = e / ld_dst;
    const int c = (int)(e - i * ld_dst);
    dst[e] = c < r_copy ? s * src[i * ld_src + c] : (T)0;
  }
}

// Frank-Wolfe factor (eq. tilde Y): Ynew[i, :r] = sY Y[i, :r],
// Ynew[i, r] = sy y_i when appending, zero padding
template <class T>
__global__ void k_fw_append(const T* __restrict__ Y, int ld, int r, const double* __restrict__ y,
                            T sY, double sy, T* __restrict__ Yn, int ld_new, int append,
                            int64_t n) {
  const int64_t total = n * ld_new;
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kBlock) {
    const int64_t i = e / ld_new;
    const int c = (int)(e - i * ld_new);
    T val = (T)0;
    if (c < r) val = sY * Y[i * ld + c];
    else if (append && c == r) val = (T)(sy * y[i]);
    Yn[e] = val;
  }
}

// m-length FP64 vectors: op 0: a = b + s c; op 1: red = <b, c>; op 2: red = |b|^2
struct OpDvec {
  int op; double* a; const double* b; const double* cc; double s;
  __device__ void operator()(int64_t i, double* red) const {
    if (op == 0) a[i] = b[i] + s * cc[i];
    else if (op == 1) red[0] += b[i] * cc[i];
    else red[0] += b[i] * b[i];
  }
};

__global__ void __launch_bounds__(kBlock) k_dvec(int64_t len, OpDvec op, double* partials,
                                                 unsigned* counter, double* out) {
  double red[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * kBlock)
    op(i, red);
  grid_reduce<1>(red, partials, counter, out);
}

// out = (To) in, elementwise
template <class To, class Ti>
__global__ void k_convert(int64_t len, To* __restrict__ out, const Ti* __restrict__ in) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * kBlock)
    out[i] = (To)in[i];
}

// Gram U^T U (rank trim): block b accumulates rows b*8.., stepping by the
// grid, into its own r x r partial; a second kernel sums the partials in
// block order.
constexpr int kGramAcc = 32;  // r*r <= 32 * 256, i.e. r <= 90
template <class T>
__global__ void __launch_bounds__(kBlock) k_gram_partial(const T* __restrict__ U, int ld, int r,
                                                         int64_t n, double* __restrict__ part) {
  extern __shared__ double rowbuf[];  // [8][ld]
  const int npair = r * r;
  double acc[kGramAcc];
#pragma unroll
  for (int q = 0; q < kGramAcc; ++q) acc[q] = 0.0;
  for (int64_t i0 = (int64_t)blockIdx.x * 8; i0 < n; i0 += (int64_t)gridDim.x * 8) {
    __syncthreads();
    for (int e = threadIdx.x; e < 8 * ld; e += kBlock) {
      const int64_t i = i0 + e / ld;
      rowbuf[e] = i < n ? (double)U[i * ld + (e % ld)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGramAcc; ++q) {
      const int pr = threadIdx.x + q * kBlock;
      if (pr < npair) {
        const int a = pr / r, bcol = pr % r;
        double s = 0.0;
        for (int rr = 0; rr < 8; ++rr) s += rowbuf[rr * ld + a] * rowbuf[rr * ld + bcol];
        acc[q] += s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kGramAcc; ++q) {
    const int pr = threadIdx.x + q * kBlock;
    if (pr < npair) part[(size_t)blockIdx.x * npair + pr] = acc[q];
  }
}

__global__ void k_sum_blocks(const double* __restrict__ part, int nblocks, int width,
                             double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < width; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * width + j];
    out[j] = s;
  }
}

// out[i, :k] = U[i, :r] Q (Q row-major r x k, FP64), zero padding to ld_out
template <class T>
__global__ void k_right_mult(const T* __restrict__ U, int ld, int r, const double* __restrict__ Q,
                             int k, T* __restrict__ out, int ld_out, int64_t n) {
  const int64_t total = n * ld_out;
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kBlock) {
    const int64_t i = e / ld_out;
    const int c = (int)(e - i * ld_out);
    double s = 0.0;
    if (c < k)
      for (int a = 0; a < r; ++a) s += (double)U[i * ld + a] * __ldg(&Q[a * k + c]);
    out[e] = (T)s;
  }
}

// r[0] = (src ? src[0] : 0) + *dscal + add (trace-row residual entry)
template <class T>
__global__ void k_trace_fix(T* dst, const T* src, const double* dscal, double add) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    dst[0] = (T)((src ? (double)src[0] : 0.0) + dscal[0] + add);
}

// run the statements with T the factor element type of the handle
#define HL_BY_TYPE(c, ...)                                    \
  do {                                                        \
    if ((c)->opt.precision == HALLAR_MIXED) {                 \
      using T = float;                                        \
      __VA_ARGS__;                                            \
    } else {                                                  \
      using T = double;                                       \
      __VA_ARGS__;                                            \
    }                                                         \
  } while (0)

}  // namespace

void launch_scale(Ctx* c, void* U, int ld, double s) {
  const int64_t ne = c->P.n * (int64_t)ld;
  HL_BY_TYPE(c, run_stream<T, 0>(c, ne, OpScale<T>{{}, (T*)U, (T)s}, -1));
}

void launch_norm2(Ctx* c, const void* U, int ld, int slot) {
  const int64_t ne = c->P.n * (int64_t)ld;
  HL_BY_TYPE(c, run_stream<T, 1>(c, ne, OpNorm2<T>{{}, (const T*)U}, slot));
}

void launch_trace_fix(Ctx* c, void* r, const void* src, const double* dscal, double add) {
  const int64_t m = c->P.m;
  HL_BY_TYPE(c, k_trace_fix<T><<<1, 32, 0, c->stream>>>(
                    (T*)r + (m - 1), src ? (const T*)src + (m - 1) : nullptr, dscal, add));
  HL_CHECK_LAUNCH(c);
}

void launch_to_factor_type(Ctx* c, int64_t len, void* out, const double* in) {
  const int grid = grid_for(c, len, kBlock * 4);
  HL_BY_TYPE(c, k_convert<T, double><<<grid, kBlock, 0, c->stream>>>(len, (T*)out, in));
  HL_CHECK_LAUNCH(c);
}

void launch_to_double(Ctx* c, int64_t len, double* out, const void* in) {
  const int grid = grid_for(c, len, kBlock * 4);
  HL_BY_TYPE(c, k_convert<double, T><<<grid, kBlock, 0, c->stream>>>(len, out, (const T*)in));
  HL_CHECK_LAUNCH(c);
}

void launch_pad_copy(Ctx* c, const void* src, int ld_src, void* dst, int ld_dst, int r_copy,
                     double scale_src) {
  const int64_t total = c->P.n * (int64_t)ld_dst;
  const int grid = grid_for(c, total, kBlock * 4);
  HL_BY_TYPE(c, k_pad_copy<T><<<grid, kBlock, 0, c->stream>>>((const T*)src, ld_src, (T*)dst,
                                                             ld_dst, r_copy, c->P.n,
                                                             (T)scale_src));
  HL_CHECK_LAUNCH(c);
}

void launch_fw_append(Ctx* c, const void* Y, int ld, int r, const double* y, double sY, double sy,
                      void* Ynew, int ld_new, int append) {
  const int64_t total = c->P.n * (int64_t)ld_new;
  const int grid = grid_for(c, total, kBlock * 4);
  HL_BY_TYPE(c, k_fw_append<T><<<grid, kBlock, 0, c->stream>>>((const T*)Y, ld, r, y, (T)sY, sy,
                                                              (T*)Ynew, ld_new, append, c->P.n));
  HL_CHECK_LAUNCH(c);
}

void launch_dvec(Ctx* c, int op, int64_t len, double* a, const double* b, const double* cc,
                 double s, int slot) {
  const int grid = grid_for(c, len, kBlock * 4);
  k_dvec<<<grid, kBlock, 0, c->stream>>>(len, OpDvec{op, a, b, cc, s}, c->red.partials,
                                         c->red.counter,
                                         c->d_scal + (slot >= 0 ? slot : S_VEC2 + 7));
  HL_CHECK_LAUNCH(c);
}

void launch_gram(Ctx* c, const void* U, int ld, int r, double* G) {
  if (r * r > kGramAcc * kBlock) fail(HALLAR_EINVAL, "rank trim supports ranks up to 90");
  // the float factor of the mixed form: on the tensor cores (gram_tc.cu);
  // FP64 factors keep the FP64 CUDA-core sum (B300's FP64 tensor rate is low)
  if (c->opt.precision == HALLAR_MIXED) {
    launch_gram_tc(c, U, ld, r, G);
    return;
  }
  int grid = grid_for(c, c->P.n, 8 * 8);
  if (grid > 512) grid = 512;
  double* part = (double*)ensure_buffer(c, &c->gram_part, &c->gram_part_bytes,
                                        (size_t)grid * r * r * sizeof(double));
  const size_t smem = (size_t)8 * ld * sizeof(double);
  HL_BY_TYPE(c, k_gram_partial<T><<<grid, kBlock, smem, c->stream>>>((const T*)U, ld, r, c->P.n,
                                                                     part));
  HL_CHECK_LAUNCH(c);
  k_sum_blocks<<<(r * r + 127) / 128, 128, 0, c->stream>>>(part, grid, r * r, G);
  HL_CHECK_LAUNCH(c);
}

void launch_right_mult(Ctx* c, const void* U, int ld, int r, const double* Q, int k, void* out,
                       int ld_out) {
  const int64_t total = c->P.n * (int64_t)ld_out;
  const int grid = grid_for(c, total, kBlock * 4);
  HL_BY_TYPE(c, k_right_mult<T><<<grid, kBlock, 0, c->stream>>>((const T*)U, ld, r, Q, k, (T*)out,
                                                               ld_out, c->P.n));
  HL_CHECK_LAUNCH(c);
}

}  // namespace hallar
