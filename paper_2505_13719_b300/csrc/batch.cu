// Batched operators: the fused constraint map + shift + SpMM of many uneven
// instances in one launch over a segmented (stacked) merged CSR.
//
// Layout.  Instance k owns rows [row_off[k], row_off[k+1]) of the stacked
// factor and constraints [cons_off[k], cons_off[k+1]).  The merged CSR of
// every instance (hallar_internal.cuh) is stacked with global row indices in
// col and global constraint indices in code; a diagonal-family row carries
// its constraint in diag_cons[i] (else -1), so one kernel serves Max-Cut
// rows (diagonal constraint plus C entries) and completion or edge rows
// (pair constraints) side by side; inst_of_row[i] gives the row's penalty.
//
// The row kernel is the thread mapping of k_grad (a group of G lanes per
// row, K 16-byte chunks per lane, edge metadata loaded once per batch of
// edges).  Each row writes its four partial sums (C.UU^T part, p.r, r.r and
// the rounding magnitude) to rowpart; one block per instance then sums its
// rows in a fixed order, so the per-instance values do not depend on
// scheduling.  The shape (G, K) for a width is fixed on the first call:
// either the rule of the single-instance kernels or the fastest candidate
// timed on the call's own data (the autotuner).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {
namespace {

template <int G>
constexpr int kEdgeBatchB = G < 4 ? G : 4;

struct BatchArgs {
  int64_t n;  // stacked rows
  int ld;
  const int* __restrict__ rowptr;
  const int* __restrict__ col;
  const int* __restrict__ code;
  const int* __restrict__ diag_cons;
  const int* __restrict__ inst_of_row;
  const void* __restrict__ cval;   // T
  const void* __restrict__ cdiag;  // T
  const void* __restrict__ b;      // T
  const void* __restrict__ p;      // T
  const void* __restrict__ beta;   // T [count]
  const void* __restrict__ U;      // T [n x ld]
  void* __restrict__ W;            // T [n x ld]
  void* __restrict__ resid;        // T [m] or null
  void* __restrict__ rowpart;      // T [n x 4]
};

template <class T, int G, int K>
__global__ void __launch_bounds__(kBlock) k_batch_grad(BatchArgs a) {
  constexpr int VEC = V16<T>::N;
  const T* __restrict__ U = static_cast<const T*>(a.U);
  T* __restrict__ W = static_cast<T*>(a.W);
  const T* __restrict__ cval = static_cast<const T*>(a.cval);
  const T* __restrict__ cdiag = static_cast<const T*>(a.cdiag);
  const T* __restrict__ bv = static_cast<const T*>(a.b);
  const T* __restrict__ pv = static_cast<const T*>(a.p);
  const T* __restrict__ betav = static_cast<const T*>(a.beta);
  T* __restrict__ resid = static_cast<T*>(a.resid);
  T* __restrict__ rowpart = static_cast<T*>(a.rowpart);
  const int lane_g = threadIdx.x & (G - 1);
  const unsigned gmask = group_mask<G>();
  const int64_t ngroups = (int64_t)gridDim.x * (kBlock / G);
  const int nch = a.ld / VEC;
  for (int64_t i = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / G; i < a.n; i += ngroups) {
    const T beta = betav[a.inst_of_row[i]];
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
    const T nrm = group_sum<G>(nrm_l, gmask);
    const T cdi = cdiag[i];
    T dcoef = cdi;
    T pr = (T)0, rr = (T)0, mag = (T)0;  // lane 0's row partials
    const int dc = a.diag_cons[i];
    if (dc >= 0) {
      // diagonal constraint: A.UU^T = |U_i|^2
      const T r = nrm - bv[dc];
      const T pl = pv[dc];
      const T ps = tfma(beta, r, pl);
      dcoef += ps;
      pr = pl * r;
      rr = r * r;
      mag = tabs(ps) * nrm;
      if (resid && lane_g == 0) resid[dc] = r;
    }
    const int e0 = a.rowptr[i], e1 = a.rowptr[i + 1];
    T cdot_l = (T)0;
    for (int eb = e0; eb < e1; eb += kEdgeBatchB<G>) {
      const int cnt = min(kEdgeBatchB<G>, e1 - eb);
      int col_t = 0, code_t = 0;
      T cv_t = (T)0;
      if (lane_g < cnt) {
        col_t = a.col[eb + lane_g];
        cv_t = cval[eb + lane_g];
        code_t = a.code[eb + lane_g];
      }
#pragma unroll
      for (int t = 0; t < kEdgeBatchB<G>; ++t) {
        const T cv = group_bcast<G>(cv_t, t, gmask);
        const int cd = group_bcast<G>(code_t, t, gmask);
        const int64_t j = group_bcast<G>(col_t, t, gmask);
        if (t >= cnt) continue;  // uniform over the group
        T uj[K][VEC];
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
        T coef;
        if (cd == kNoCons) {
          coef = cv;
#pragma unroll
          for (int k = 0; k < K; ++k)
#pragma unroll
            for (int v = 0; v < VEC; ++v) cdot_l = tfma(coef * u[k][v], uj[k][v], cdot_l);
        } else {
          // pair constraint l: A_l.UU^T = <U_i, U_j>
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
          if (owner) {
            pr += pl * r;
            rr += r * r;
            mag += tabs(ps) * tabs(dot);
            if (resid && lane_g == 0) resid[l] = r;
          }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[k][v] = tfma(coef, uj[k][v], acc[k][v]);
      }
    }
    const T cdot = group_sum<G>(cdot_l, gmask);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int ch = lane_g + k * G;
      if (ch < nch) {
        T w[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) w[v] = tfma(dcoef, u[k][v], acc[k][v]);
        store_chunk<T>(W, rowoff + ch * VEC, w);
      }
    }
    if (lane_g == 0) {
      rowpart[i * 4 + 0] = tfma(cdi, nrm, cdot);
      rowpart[i * 4 + 1] = pr;
      rowpart[i * 4 + 2] = rr;
      rowpart[i * 4 + 3] = mag + tabs(cdot) + tabs(cdi) * nrm;
    }
  }
}

// per-instance sums of the row partials, in a fixed order: block k owns
// instance k; g_k = T0 + p.r + beta_k/2 r.r, out[k] = [T0, p.r, r.r, mag]
template <class T>
__global__ void __launch_bounds__(kBlock) k_batch_reduce(const T* __restrict__ rowpart,
                                                         const int64_t* __restrict__ row_off,
                                                         const double* __restrict__ beta,
                                                         double* __restrict__ out,
                                                         double* __restrict__ g) {
  __shared__ double sh[4][kBlock / 32];
  const int k = blockIdx.x;
  const int64_t r0 = row_off[k], r1 = row_off[k + 1];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kBlock) {
#pragma unroll
    for (int s = 0; s < 4; ++s) v[s] += (double)rowpart[i * 4 + s];
  }
  block_sum<4>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < 4; ++s) out[(size_t)k * 4 + s] = v[s];
    g[k] = v[0] + v[1] + 0.5 * beta[k] * v[2];
  }
}

template <class To, class Ti>
__global__ void k_batch_convert(int64_t len, To* __restrict__ out, const Ti* __restrict__ in) {
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * kBlock)
    out[i] = (To)in[i];
}

struct BShape {
  int G, K;
};

// shapes with a kernel instantiation; the candidates for a row of nch
// 16-byte chunks, the built-in rule's choice first
std::vector<BShape> candidates(int nch) {
  if (nch <= 5) {
    std::vector<BShape> c{{1, nch}};
    if ((nch + 1) / 2 <= 3 && nch > 1) c.push_back({2, (nch + 1) / 2});
    if (nch <= 4) c.push_back({4, 1});
    c.push_back({8, 1});
    return c;
  }
  if (nch <= 8) return {{4, 2}, {8, 1}};
  if (nch <= 16) return {{16, 1}, {8, 2}};
  if (nch <= 32) return {{32, 1}};
  if (nch <= 64) return {{32, 2}};
  return {{32, 4}};
}

#define HL_BATCH_SHAPES(G_, K_, ...)                                               \
  switch ((G_) * 10 + (K_)) {                                                      \
    case 11: { constexpr int G = 1, K = 1; __VA_ARGS__; } break;                   \
    case 12: { constexpr int G = 1, K = 2; __VA_ARGS__; } break;                   \
    case 13: { constexpr int G = 1, K = 3; __VA_ARGS__; } break;                   \
    case 14: { constexpr int G = 1, K = 4; __VA_ARGS__; } break;                   \
    case 15: { constexpr int G = 1, K = 5; __VA_ARGS__; } break;                   \
    case 21: { constexpr int G = 2, K = 1; __VA_ARGS__; } break;                   \
    case 22: { constexpr int G = 2, K = 2; __VA_ARGS__; } break;                   \
    case 23: { constexpr int G = 2, K = 3; __VA_ARGS__; } break;                   \
    case 41: { constexpr int G = 4, K = 1; __VA_ARGS__; } break;                   \
    case 42: { constexpr int G = 4, K = 2; __VA_ARGS__; } break;                   \
    case 81: { constexpr int G = 8, K = 1; __VA_ARGS__; } break;                   \
    case 82: { constexpr int G = 8, K = 2; __VA_ARGS__; } break;                   \
    case 161: { constexpr int G = 16, K = 1; __VA_ARGS__; } break;                 \
    case 321: { constexpr int G = 32, K = 1; __VA_ARGS__; } break;                 \
    case 322: { constexpr int G = 32, K = 2; __VA_ARGS__; } break;                 \
    case 324: { constexpr int G = 32, K = 4; __VA_ARGS__; } break;                 \
    default: throw Err{HALLAR_EINVAL, "batch: no kernel for this shape"};          \
  }

thread_local std::string g_batch_create_error;

bool is_dev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace hallar

using namespace hallar;

struct hallar_batch {
  int count = 0;
  int precision = HALLAR_FP64;
  bool autotune = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, num_sms = 0;
  std::vector<int64_t> row_off, cons_off;
  int64_t n_total = 0, m_total = 0, nnz_total = 0;
  // device arrays
  int *rowptr = nullptr, *col = nullptr, *code = nullptr, *diag_cons = nullptr,
      *inst_of_row = nullptr;
  void *cval = nullptr, *cdiag = nullptr, *b = nullptr;  // factor type
  int64_t* d_row_off = nullptr;
  void *p_t = nullptr, *beta_t = nullptr;                 // factor type staging
  double *beta_d = nullptr, *p_d = nullptr, *out = nullptr, *g_d = nullptr, *resid_d = nullptr;
  void* rowpart = nullptr;
  void *U_pad = nullptr, *W_pad = nullptr, *resid_t = nullptr;
  int pad_ld = 0;
  std::vector<void*> owned;
  std::map<int, std::pair<BShape, bool>> shapes;  // ld -> (shape, tuned)
  std::string last_error;
};

namespace {

size_t esz(const hallar_batch* bt) { return bt->precision == HALLAR_MIXED ? 4 : 8; }

void* balloc(hallar_batch* bt, size_t bytes) {
  void* p = nullptr;
  HL_CUDA(cudaMallocAsync(&p, std::max<size_t>(bytes, 16), bt->stream));
  bt->owned.push_back(p);
  return p;
}

template <class T>
void* upload_as(hallar_batch* bt, const std::vector<double>& v) {
  std::vector<T> t(v.begin(), v.end());
  void* d = balloc(bt, t.size() * sizeof(T));
  if (!t.empty())
    HL_CUDA(cudaMemcpyAsync(d, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice,
                            bt->stream));
  // t is staged by the call (pageable source) before it returns
  return d;
}

template <class V>
V* upload_vec(hallar_batch* bt, const std::vector<V>& v) {
  V* d = static_cast<V*>(balloc(bt, v.size() * sizeof(V)));
  if (!v.empty())
    HL_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice,
                            bt->stream));
  return d;
}

void release_batch(hallar_batch* bt) {
  if (!bt) return;
  for (void* p : bt->owned) cudaFreeAsync(p, bt->stream);
  bt->owned.clear();
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  if (bt->own_stream && bt->stream) cudaStreamDestroy(bt->stream);
  delete bt;
}

template <class T>
void launch_batch(hallar_batch* bt, BShape s, int ld, const void* U, void* W, bool want_resid) {
  BatchArgs a;
  a.n = bt->n_total;
  a.ld = ld;
  a.rowptr = bt->rowptr;
  a.col = bt->col;
  a.code = bt->code;
  a.diag_cons = bt->diag_cons;
  a.inst_of_row = bt->inst_of_row;
  a.cval = bt->cval;
  a.cdiag = bt->cdiag;
  a.b = bt->b;
  a.p = bt->p_t;
  a.beta = bt->beta_t;
  a.U = U;
  a.W = W;
  a.resid = want_resid ? bt->resid_t : nullptr;
  a.rowpart = bt->rowpart;
  HL_BATCH_SHAPES(s.G, s.K, {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_grad<T, G, K>, kBlock, 0) !=
            cudaSuccess || nb < 1) {
      cudaGetLastError();
      nb = 1;
    }
    int64_t grid = (bt->n_total + (kBlock / G) - 1) / (kBlock / G);
    grid = std::min<int64_t>(grid, (int64_t)nb * bt->num_sms);
    grid = std::max<int64_t>(grid, 1);
    k_batch_grad<T, G, K><<<(int)grid, kBlock, 0, bt->stream>>>(a);
  });
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Err{HALLAR_ECUDA, cudaGetErrorString(e)};
}

template <class F>
hallar_status batch_guard(hallar_batch* bt, F&& f) {
  if (!bt) return HALLAR_EINVAL;
  try {
    HL_CUDA(cudaSetDevice(bt->device));
    bt->last_error.clear();
    return f();
  } catch (const Err& e) {
    bt->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    bt->last_error = "host allocation failed";
    return HALLAR_ENOMEM;
  }
}

}  // namespace

extern "C" {

hallar_status hallar_batch_create(int32_t count, const hallar_request* problems,
                                  int32_t precision, int32_t autotune, void* stream,
                                  hallar_batch_t* out) {
  g_batch_create_error.clear();
  if (!out) {
    g_batch_create_error = "out is NULL";
    return HALLAR_EINVAL;
  }
  *out = nullptr;
  if (count < 1 || !problems || (precision != HALLAR_FP64 && precision != HALLAR_MIXED)) {
    g_batch_create_error = "count, problems or precision invalid";
    return HALLAR_EINVAL;
  }
  hallar_batch* bt = new (std::nothrow) hallar_batch();
  if (!bt) return HALLAR_ENOMEM;
  try {
    bt->count = count;
    bt->precision = precision;
    bt->autotune = autotune != 0;
    HL_CUDA(cudaGetDevice(&bt->device));
    HL_CUDA(cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, bt->device));
    if (stream) {
      bt->stream = (cudaStream_t)stream;
    } else {
      HL_CUDA(cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking));
      bt->own_stream = true;
    }
    // merge every instance on the host, then stack with global indices
    std::vector<int32_t> rowptr{0}, col, code, diag_cons, inst_of_row;
    std::vector<double> val, cdiag, b;
    bt->row_off.assign(1, 0);
    bt->cons_off.assign(1, 0);
    for (int k = 0; k < count; ++k) {
      const hallar_request& q = problems[k];
      HostProblem P;
      try {
        merge_problem(P, q.n, q.n1, q.C_rowptr, q.C_col, q.C_val, q.C_J, q.C_I, q.family,
                      q.m_pairs, q.cons_i, q.cons_j, q.has_trace_row, q.b, q.tau2);
      } catch (const Err& e) {
        throw Err{e.st, "instance " + std::to_string(k) + ": " + e.msg};
      }
      if (P.has_trace || P.C_J != 0.0)
        throw Err{HALLAR_EINVAL, "instance " + std::to_string(k) +
                                     ": the batch takes no trace row and no C_J"};
      const int64_t r0 = bt->row_off.back(), c0 = bt->cons_off.back();
      if (r0 + P.n >= (int64_t)INT32_MAX || c0 + P.m >= (int64_t)INT32_MAX ||
          (int64_t)col.size() + P.nnz >= (int64_t)INT32_MAX)
        throw Err{HALLAR_EINVAL, "batch too large for 32-bit indices"};
      const int64_t e0 = (int64_t)col.size();
      for (int64_t i = 0; i < P.n; ++i) {
        for (int64_t e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e) {
          col.push_back((int32_t)(P.col[e] + r0));
          if (P.fam == FAM_DIAG) {
            code.push_back(kNoCons);
          } else {
            const int32_t cd = P.code[e];
            code.push_back(cd == kNoCons ? kNoCons
                                         : (cd >= 0 ? (int32_t)(cd + c0) : (int32_t)(cd - c0)));
          }
          val.push_back(P.val.empty() ? 0.0 : P.val[e]);
        }
        rowptr.push_back((int32_t)(e0 + P.rowptr[i + 1]));
        diag_cons.push_back(P.fam == FAM_DIAG ? (int32_t)(c0 + i) : -1);
        inst_of_row.push_back(k);
        cdiag.push_back(P.cdiag[i]);
      }
      b.insert(b.end(), P.b.begin(), P.b.end());
      bt->row_off.push_back(r0 + P.n);
      bt->cons_off.push_back(c0 + P.m);
    }
    bt->n_total = bt->row_off.back();
    bt->m_total = bt->cons_off.back();
    bt->nnz_total = (int64_t)col.size();
    bt->rowptr = upload_vec(bt, rowptr);
    bt->col = upload_vec(bt, col);
    bt->code = upload_vec(bt, code);
    bt->diag_cons = upload_vec(bt, diag_cons);
    bt->inst_of_row = upload_vec(bt, inst_of_row);
    bt->d_row_off = upload_vec(bt, bt->row_off);
    const bool mixed = precision == HALLAR_MIXED;
    bt->cval = mixed ? upload_as<float>(bt, val) : upload_as<double>(bt, val);
    bt->cdiag = mixed ? upload_as<float>(bt, cdiag) : upload_as<double>(bt, cdiag);
    bt->b = mixed ? upload_as<float>(bt, b) : upload_as<double>(bt, b);
    const size_t es = esz(bt);
    bt->p_t = balloc(bt, (size_t)bt->m_total * es);
    bt->beta_t = balloc(bt, (size_t)count * es);
    bt->beta_d = (double*)balloc(bt, (size_t)count * sizeof(double));
    bt->p_d = (double*)balloc(bt, (size_t)bt->m_total * sizeof(double));
    bt->out = (double*)balloc(bt, (size_t)count * 4 * sizeof(double));
    bt->g_d = (double*)balloc(bt, (size_t)count * sizeof(double));
    bt->resid_d = (double*)balloc(bt, (size_t)bt->m_total * sizeof(double));
    bt->resid_t = balloc(bt, (size_t)bt->m_total * es);
    bt->rowpart = balloc(bt, (size_t)bt->n_total * 4 * es);
    HL_CUDA(cudaStreamSynchronize(bt->stream));
  } catch (const Err& e) {
    g_batch_create_error = e.msg;
    release_batch(bt);
    return e.st;
  } catch (const std::bad_alloc&) {
    g_batch_create_error = "host allocation failed";
    release_batch(bt);
    return HALLAR_ENOMEM;
  }
  *out = bt;
  return HALLAR_OK;
}

hallar_status hallar_batch_layout(hallar_batch_t bt, int64_t* row_off, int64_t* cons_off,
                                  int64_t* n_total, int64_t* m_total) {
  if (!bt) return HALLAR_EINVAL;
  if (row_off) std::memcpy(row_off, bt->row_off.data(), bt->row_off.size() * sizeof(int64_t));
  if (cons_off)
    std::memcpy(cons_off, bt->cons_off.data(), bt->cons_off.size() * sizeof(int64_t));
  if (n_total) *n_total = bt->n_total;
  if (m_total) *m_total = bt->m_total;
  return HALLAR_OK;
}

hallar_status hallar_batch_grad(hallar_batch_t bt, const void* U, int32_t r, const double* p,
                                const double* beta, void* W, double* g, double* resid) {
  return batch_guard(bt, [&]() -> hallar_status {
    if (!U || !p || !beta || !W || !g || r < 1 || r > 256)
      throw Err{HALLAR_EINVAL, "hallar_batch_grad: bad argument"};
    const bool mixed = bt->precision == HALLAR_MIXED;
    const size_t es = esz(bt);
    const int vec = mixed ? 4 : 2;
    const int ld = (r + vec - 1) / vec * vec;
    cudaStream_t s = bt->stream;
    const int64_t n = bt->n_total, m = bt->m_total;
    // padded factor buffers (pad columns stay zero: copies write r columns)
    if (bt->pad_ld < ld) {
      bt->U_pad = balloc(bt, (size_t)n * ld * es);
      bt->W_pad = balloc(bt, (size_t)n * ld * es);
      HL_CUDA(cudaMemsetAsync(bt->U_pad, 0, (size_t)n * ld * es, s));
      bt->pad_ld = ld;
    }
    const void* Ud = U;
    void* Wd = W;
    const bool direct = ld == r && is_dev(U) && is_dev(W) && ((uintptr_t)U % 16) == 0 &&
                        ((uintptr_t)W % 16) == 0;
    if (!direct) {
      HL_CUDA(cudaMemcpy2DAsync(bt->U_pad, (size_t)ld * es, U, (size_t)r * es, (size_t)r * es,
                                (size_t)n, cudaMemcpyDefault, s));
      Ud = bt->U_pad;
      Wd = bt->W_pad;
    }
    // multipliers and penalties in the factor type (and beta in double)
    HL_CUDA(cudaMemcpyAsync(bt->p_d, p, (size_t)m * sizeof(double), cudaMemcpyDefault, s));
    HL_CUDA(cudaMemcpyAsync(bt->beta_d, beta, (size_t)bt->count * sizeof(double),
                            cudaMemcpyDefault, s));
    const int gp = (int)std::min<int64_t>((m + kBlock - 1) / kBlock, 4LL * bt->num_sms);
    const int gb = (int)std::min<int64_t>((bt->count + kBlock - 1) / kBlock, 4LL * bt->num_sms);
    if (mixed) {
      k_batch_convert<float, double><<<std::max(gp, 1), kBlock, 0, s>>>(m, (float*)bt->p_t, bt->p_d);
      k_batch_convert<float, double><<<std::max(gb, 1), kBlock, 0, s>>>(bt->count,
                                                                         (float*)bt->beta_t,
                                                                         bt->beta_d);
    } else {
      HL_CUDA(cudaMemcpyAsync(bt->p_t, bt->p_d, (size_t)m * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
      HL_CUDA(cudaMemcpyAsync(bt->beta_t, bt->beta_d, (size_t)bt->count * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    }
    // the kernel shape for this width: fixed on first use
    auto it = bt->shapes.find(ld);
    if (it == bt->shapes.end()) {
      const std::vector<BShape> cand = candidates(ld / vec);
      BShape best = cand[0];
      bool tuned = false;
      if (bt->autotune && cand.size() > 1) {
        cudaEvent_t e0, e1;
        HL_CUDA(cudaEventCreate(&e0));
        HL_CUDA(cudaEventCreate(&e1));
        float best_ms = 0.0f;
        for (size_t c = 0; c < cand.size(); ++c) {
          if (mixed) launch_batch<float>(bt, cand[c], ld, Ud, Wd, false);  // warm-up
          else launch_batch<double>(bt, cand[c], ld, Ud, Wd, false);
          HL_CUDA(cudaEventRecord(e0, s));
          for (int rep = 0; rep < 3; ++rep) {
            if (mixed) launch_batch<float>(bt, cand[c], ld, Ud, Wd, false);
            else launch_batch<double>(bt, cand[c], ld, Ud, Wd, false);
          }
          HL_CUDA(cudaEventRecord(e1, s));
          HL_CUDA(cudaEventSynchronize(e1));
          float ms = 0.0f;
          HL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          // a candidate replaces the rule's choice only when 5 % faster
          if (c == 0 || ms < 0.95f * best_ms) {
            best_ms = ms;
            best = cand[c];
          }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tuned = true;
      }
      it = bt->shapes.emplace(ld, std::make_pair(best, tuned)).first;
    }
    if (mixed) launch_batch<float>(bt, it->second.first, ld, Ud, Wd, resid != nullptr);
    else launch_batch<double>(bt, it->second.first, ld, Ud, Wd, resid != nullptr);
    if (mixed)
      k_batch_reduce<float><<<bt->count, kBlock, 0, s>>>((const float*)bt->rowpart, bt->d_row_off,
                                                          bt->beta_d, bt->out, bt->g_d);
    else
      k_batch_reduce<double><<<bt->count, kBlock, 0, s>>>((const double*)bt->rowpart,
                                                           bt->d_row_off, bt->beta_d, bt->out,
                                                           bt->g_d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Err{HALLAR_ECUDA, cudaGetErrorString(e)};
    if (!direct)
      HL_CUDA(cudaMemcpy2DAsync(W, (size_t)r * es, bt->W_pad, (size_t)ld * es, (size_t)r * es,
                                (size_t)n, cudaMemcpyDefault, s));
    HL_CUDA(cudaMemcpyAsync(g, bt->g_d, (size_t)bt->count * sizeof(double), cudaMemcpyDefault,
                            s));
    if (resid) {
      if (mixed) {
        k_batch_convert<double, float><<<std::max(gp, 1), kBlock, 0, s>>>(m, bt->resid_d,
                                                                           (const float*)bt->resid_t);
        HL_CUDA(cudaMemcpyAsync(resid, bt->resid_d, (size_t)m * sizeof(double),
                                cudaMemcpyDefault, s));
      } else {
        HL_CUDA(cudaMemcpyAsync(resid, bt->resid_t, (size_t)m * sizeof(double),
                                cudaMemcpyDefault, s));
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) throw Err{HALLAR_ECUDA, cudaGetErrorString(e)};
    HL_CUDA(cudaStreamSynchronize(s));
    return HALLAR_OK;
  });
}

hallar_status hallar_batch_shape(hallar_batch_t bt, int32_t r, int32_t* G, int32_t* K,
                                 int32_t* tuned) {
  if (!bt || r < 1 || r > 256) return HALLAR_EINVAL;
  const int vec = bt->precision == HALLAR_MIXED ? 4 : 2;
  const int ld = (r + vec - 1) / vec * vec;
  auto it = bt->shapes.find(ld);
  if (it == bt->shapes.end()) {
    bt->last_error = "no hallar_batch_grad call with this width yet";
    return HALLAR_EINVAL;
  }
  if (G) *G = it->second.first.G;
  if (K) *K = it->second.first.K;
  if (tuned) *tuned = it->second.second ? 1 : 0;
  return HALLAR_OK;
}

void hallar_batch_destroy(hallar_batch_t bt) {
  if (!bt) return;
  cudaSetDevice(bt->device);
  release_batch(bt);
}

const char* hallar_batch_last_error(hallar_batch_t bt) {
  if (!bt) return g_batch_create_error.c_str();
  return bt->last_error.c_str();
}

}  // extern "C"
