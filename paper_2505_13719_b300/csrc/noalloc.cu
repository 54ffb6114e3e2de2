// Allocation-free fused gradient for the diagonal (Max-Cut) constraint family.
//
// The regular entry points run through a handle that owns device buffers it
// allocates with cudaMalloc.  Some callers cannot allow that: applications
// that hand out device memory only from their own pool or arena and account
// for every byte, and hot paths where an allocation (or the device-wide
// synchronisation of a later cudaFree) would stall work queued on other
// streams.  hallar_grad_diag_noalloc serves them: the caller passes every input
// and output array, and the only scratch the kernel needs -- the per-block
// partial sums and the arrival counter of its grid reduction -- lives in the
// file-scope device array below.
//
// The array costs every GPU that loads this library kNaScratchDoubles * 8
// bytes (about 29 KB) until the process exits.  In host code its name is a
// host-side stand-in, not a device address, so the host looks the device
// address up with cudaGetSymbolAddress once per device (on the first call
// on that device, with that device current; again after the device's
// context was re-created) and passes it to the kernel.
// All calls share the array and it keeps the last call's contents: each call
// clears the arrival counter before its kernel, and calls whose kernels
// overlap on the GPU race on the array.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "device_common.cuh"
#include "../../include/hallar.h"

namespace hallar {
namespace {

constexpr int kNaMaxBlocks = 1184;                       // 8 blocks on each of 148 SMs
constexpr int kNaCounter = 3 * kNaMaxBlocks;             // index of the arrival counter
constexpr int kNaScratchDoubles = 3 * kNaMaxBlocks + 32;
constexpr int kNaMaxDevices = 64;
constexpr int kNaMaxR = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNaScratchDoubles];

struct DevState {
  double* scratch = nullptr;  // device address of g_noalloc_scratch
  int sms = 0;
  unsigned long long ctx_id = 0;  // context the address belongs to (0: unknown)
};
std::mutex g_na_mu;
DevState g_na_dev[kNaMaxDevices];

// Unique ID of the calling thread's current CUDA context, or 0 when it cannot
// be read.  A device reset or a destroyed and re-created primary context
// reloads this module at a new address; comparing context IDs tells the
// cached address is stale.  The driver calls are reached through the
// runtime's entry-point query, so the library needs no link to libcuda.
using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // under g_na_mu
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
  }
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || ctx == nullptr) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != 0) return 0;
  return id;
}

// Same arithmetic as the fused operator for the diagonal family: per row i,
// |U_i|^2, r_i = |U_i|^2 - b_i, p'_i = p_i + beta r_i, W_i = sum_j C_ij U_j +
// (C_ii + p'_i) U_i, and the sums C.UU^T, p^T r, r^T r; the last block to
// finish writes g = C.UU^T + p^T r + beta/2 r^T r to g_out.
template <int G>
__global__ void __launch_bounds__(kBlock)
    k_grad_diag_noalloc(int64_t n, int ld, const int* __restrict__ rowptr,
                        const int* __restrict__ col, const double* __restrict__ cval,
                        const double* __restrict__ cdiag, const double* __restrict__ b,
                        const double* __restrict__ p, double beta, const double* __restrict__ U,
                        double* __restrict__ W, double* __restrict__ resid,
                        double* __restrict__ scratch, double* __restrict__ g_out) {
  constexpr int VEC = 2;
  const int lane_g = threadIdx.x & (G - 1);
  const unsigned gmask = group_mask<G>();
  const int64_t ngroups = (int64_t)gridDim.x * (kBlock / G);
  const int nch = ld / VEC;
  double red[3] = {0.0, 0.0, 0.0};
  for (int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / G; i < n; i += ngroups) {
    double u[VEC] = {0.0, 0.0}, acc[VEC] = {0.0, 0.0};
    const int64_t rowoff = i * (int64_t)ld;
    if (lane_g < nch) load_chunk<double>(U, rowoff + lane_g * VEC, u);
    const double nrm = group_sum<G>(fma(u[0], u[0], u[1] * u[1]), gmask);
    const double r = nrm - b[i];
    const double ps = p[i] + beta * r;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      double uj[VEC] = {0.0, 0.0};
      if (lane_g < nch) load_chunk_l2<double>(U, (int64_t)col[e] * ld + lane_g * VEC, uj);
      const double cv = cval[e];
      acc[0] = fma(cv, uj[0], acc[0]);
      acc[1] = fma(cv, uj[1], acc[1]);
    }
    red[0] += fma(u[0], acc[0], u[1] * acc[1]);
    if (lane_g == 0) {
      red[0] += cdiag[i] * nrm;
      red[1] += p[i] * r;
      red[2] += r * r;
      if (resid) resid[i] = r;
    }
    if (lane_g < nch) {
      const double dc = cdiag[i] + ps;
      double w[VEC] = {fma(dc, u[0], acc[0]), fma(dc, u[1], acc[1])};
      store_chunk<double>(W, rowoff + lane_g * VEC, w);
    }
  }
  // deterministic grid reduction through the static scratch
  __shared__ double sh[3][kBlock / 32];
  __shared__ bool am_last;
  block_sum<3>(red, sh);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNaCounter);
  if (threadIdx.x == 0) {
    for (int s = 0; s < 3; ++s) scratch[(size_t)blockIdx.x * 3 + s] = red[s];
    __threadfence();
    am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double acc3[3] = {0.0, 0.0, 0.0};
  for (unsigned bb = threadIdx.x; bb < gridDim.x; bb += kBlock)
    for (int s = 0; s < 3; ++s) acc3[s] += __ldcg(&scratch[(size_t)bb * 3 + s]);
  block_sum<3>(acc3, sh);
  if (threadIdx.x == 0) {
    g_out[0] = acc3[0] + acc3[1] + 0.5 * beta * acc3[2];
    *counter = 0u;
  }
}

void set_err(char* buf, int len, const char* msg) {
  if (buf && len > 0) std::snprintf(buf, (size_t)len, "%s", msg);
}

}  // namespace
}  // namespace hallar

using namespace hallar;

extern "C" hallar_status hallar_grad_diag_noalloc(
    int64_t n, int32_t r, const int32_t* rowptr, const int32_t* col, const double* cval,
    const double* cdiag, const double* b, const double* p, double beta, const double* U,
    double* W, double* resid, double* g_out, void* stream, char* errbuf, int32_t errbuf_len) {
  set_err(errbuf, errbuf_len, "");
  if (n < 1 || n >= (int64_t)INT32_MAX) {
    set_err(errbuf, errbuf_len, "hallar_grad_diag_noalloc: n must be in [1, 2^31 - 1)");
    return HALLAR_EINVAL;
  }
  if (r < 2 || r > kNaMaxR || (r & 1)) {
    set_err(errbuf, errbuf_len,
            "hallar_grad_diag_noalloc: r must be even and in [2, 64] (rows of 16-byte chunks)");
    return HALLAR_EINVAL;
  }
  if (!rowptr || !col || !cval || !cdiag || !b || !p || !U || !W || !g_out ||
      !std::isfinite(beta)) {
    set_err(errbuf, errbuf_len, "hallar_grad_diag_noalloc: null array or non-finite beta");
    return HALLAR_EINVAL;
  }
  if (((uintptr_t)U % 16) != 0 || ((uintptr_t)W % 16) != 0) {
    set_err(errbuf, errbuf_len, "hallar_grad_diag_noalloc: U and W must be 16-byte aligned");
    return HALLAR_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    set_err(errbuf, errbuf_len, "hallar_grad_diag_noalloc: no usable current device");
    return HALLAR_ECUDA;
  }
  DevState st;
  {
    std::lock_guard<std::mutex> lock(g_na_mu);
    DevState& d = g_na_dev[dev];
    const unsigned long long ctx_now = current_ctx_id();
    if (d.scratch != nullptr && d.ctx_id != 0 && ctx_now != 0 && ctx_now != d.ctx_id)
      d.scratch = nullptr;  // the context was re-created: look the address up again
    if (d.scratch == nullptr) {
      // once per device (and context), with that device current: the
      // scratch's device address
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        set_err(errbuf, errbuf_len, "hallar_grad_diag_noalloc: cudaGetSymbolAddress failed");
        return HALLAR_ECUDA;
      }
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        set_err(errbuf, errbuf_len, "hallar_grad_diag_noalloc: cannot read the SM count");
        return HALLAR_ECUDA;
      }
      d.scratch = static_cast<double*>(ptr);
      d.sms = sms;
      d.ctx_id = current_ctx_id();
    }
    st = d;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the arrival counter must start at zero
  if (cudaMemsetAsync(st.scratch + kNaCounter, 0, sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    set_err(errbuf, errbuf_len, "hallar_grad_diag_noalloc: clearing the counter failed");
    return HALLAR_ECUDA;
  }
  int G = 2;
  while (G < r / 2) G <<= 1;
  const int64_t rows_per_block = kBlock / G;
  int64_t grid = (n + rows_per_block - 1) / rows_per_block;
  int64_t cap = (int64_t)st.sms * 8;
  if (cap > kNaMaxBlocks) cap = kNaMaxBlocks;
  if (grid > cap) grid = cap;
#define HL_NA_LAUNCH(GG)                                                                      \
  k_grad_diag_noalloc<GG><<<(int)grid, kBlock, 0, s>>>(n, r, rowptr, col, cval, cdiag, b, p,  \
                                                      beta, U, W, resid, st.scratch, g_out)
  switch (G) {
    case 2: HL_NA_LAUNCH(2); break;
    case 4: HL_NA_LAUNCH(4); break;
    case 8: HL_NA_LAUNCH(8); break;
    case 16: HL_NA_LAUNCH(16); break;
    default: HL_NA_LAUNCH(32); break;
  }
#undef HL_NA_LAUNCH
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(errbuf, errbuf_len, cudaGetErrorString(e));
    return HALLAR_ECUDA;
  }
  return HALLAR_OK;
}
