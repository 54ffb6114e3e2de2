// C entry points of the HALLaR library (declared in include/hallar.h):
// input validation, the merged CSR layout in HBM, host/device pointer
// staging and the error model (a status per call, a message per handle).
#include <algorithm>
#include <cmath>
#include <climits>
#include <map>
#include <mutex>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

int resident_blocks(const void* fn, int block, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::pair<const void*, int> key(fn, dev * 4096 + block);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cache[key] = nb;
  return nb;
}


void dfree(Ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->owned.begin(), c->owned.end(), p);
  if (it != c->owned.end()) c->owned.erase(it);
  cudaFreeAsync(p, c->stream);
}

namespace {
std::mutex g_pin_mu;
std::vector<double*> g_pin_free;
constexpr int kPinSlab = 64;  // blocks per pinned slab
}  // namespace

double* pinned_scalars_acquire() {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  if (g_pin_free.empty()) {
    double* slab = nullptr;
    HL_CUDA(cudaMallocHost((void**)&slab, (size_t)kPinSlab * kPinDoubles * sizeof(double)));
    for (int i = kPinSlab - 1; i >= 0; --i) g_pin_free.push_back(slab + (size_t)i * kPinDoubles);
  }
  double* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

void pinned_scalars_release(double* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_pin_free.push_back(p);
}

void* ensure_buffer(Ctx* c, void** buf, size_t* cur, size_t bytes) {
  if (*buf && *cur >= bytes) return *buf;
  if (*buf) dfree(c, *buf);
  *buf = nullptr;
  *cur = 0;
  *buf = dalloc<unsigned char>(c, bytes);
  *cur = bytes;
  return *buf;
}

void sync(Ctx* c) {
  HL_CUDA(cudaStreamSynchronize(c->stream));
  if (!c->prof_pending.empty()) prof_resolve(c);
}

void fetch_scalars(Ctx* c, int first, int count) {
  HL_CUDA(cudaMemcpyAsync(c->h_scal + first, c->d_scal + first, count * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream));
  sync(c);
}

int prof_begin(Ctx* c, int cls, OpBytes bytes) {
  if (!c->prof_on || c->capturing) return -1;
  if (c->prof_seen[cls]++ % c->prof_every != 0) return -1;  // not sampled
  c->prof_bytes[cls] += bytes.alg;
  c->prof_bytes_pad[cls] += bytes.pad;
  // the pool is reused: pending pair q uses events 2q and 2q + 1
  const size_t idx = c->prof_pending.size();  // two entries per pending pair
  while (c->prof_pool.size() < idx + 2) {
    cudaEvent_t e;
    HL_CUDA(cudaEventCreate(&e));
    c->prof_pool.push_back(e);
  }
  HL_CUDA(cudaEventRecord(c->prof_pool[idx], c->stream));
  c->prof_pending.push_back(cls);
  c->prof_pending.push_back((int)idx);
  return (int)idx;
}

void prof_end(Ctx* c, int token) {
  if (token < 0) return;
  HL_CUDA(cudaEventRecord(c->prof_pool[token + 1], c->stream));
}

void prof_resolve(Ctx* c) {
  for (size_t q = 0; q + 1 < c->prof_pending.size(); q += 2) {
    const int cls = c->prof_pending[q], idx = c->prof_pending[q + 1];
    float ms = 0.0f;
    HL_CUDA(cudaEventSynchronize(c->prof_pool[idx + 1]));
    HL_CUDA(cudaEventElapsedTime(&ms, c->prof_pool[idx], c->prof_pool[idx + 1]));
    c->prof_ms[cls] += ms;
    c->prof_n[cls] += 1;
  }
  c->prof_pending.clear();
}

namespace {

thread_local std::string g_create_error;

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
T* upload(Ctx* c, const T* host, size_t count) {
  T* d = dalloc<T>(c, count);
  // from pageable memory the call returns once the data is staged, so the
  // caller's array may be released afterwards
  if (count)
    HL_CUDA(cudaMemcpyAsync(d, host, count * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return d;
}

bool finite_all(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

// Validates the data and builds the merged CSR on the host (layout in
// hallar_internal.cuh); throws Err on invalid input.
void merge_problem(HostProblem& P, int64_t n, int64_t n1, const int64_t* rp, const int32_t* ci,
                   const double* cv, double C_J, double C_I, int family, int64_t m_pairs,
                   const int32_t* pi, const int32_t* pj, int has_trace, const double* b,
                   double tau2) {
  if (n <= 0 || n >= (int64_t)INT32_MAX) fail(HALLAR_EINVAL, "n must be in [1, 2^31 - 1)");
  if (family < 0 || family > 2) fail(HALLAR_EINVAL, "unknown constraint family");
  if (!(tau2 > 0.0) || !std::isfinite(tau2)) fail(HALLAR_EINVAL, "tau2 must be positive and finite");
  if (!std::isfinite(C_J) || !std::isfinite(C_I)) fail(HALLAR_EINVAL, "C_J / C_I not finite");
  if (!b) fail(HALLAR_EINVAL, "b is NULL");
  int64_t m;
  if (family == HALLAR_DIAG) {
    if (m_pairs != 0 || has_trace) fail(HALLAR_EINVAL, "DIAG family takes no pairs and no trace row");
    m = n;
  } else {
    if (m_pairs < 0 || m_pairs >= (int64_t)INT32_MAX - 1) fail(HALLAR_EINVAL, "m_pairs out of range");
    if (m_pairs > 0 && (!pi || !pj)) fail(HALLAR_EINVAL, "cons_i / cons_j NULL");
    if (family == HALLAR_OBSERVED && (n1 <= 0 || n1 >= n)) fail(HALLAR_EINVAL, "n1 must be in (0, n)");
    m = m_pairs + (has_trace ? 1 : 0);
    if (m == 0) fail(HALLAR_EINVAL, "no constraints");
  }
  if (!finite_all(b, (size_t)m)) fail(HALLAR_EINVAL, "b has a non-finite entry");
  // ---- C: row pointers, indices, values, symmetry ----
  int64_t nnzC = 0;
  if (rp) {
    if (rp[0] != 0) fail(HALLAR_EINVAL, "C_rowptr[0] must be 0");
    for (int64_t i = 0; i < n; ++i)
      if (rp[i + 1] < rp[i]) fail(HALLAR_EINVAL, "C_rowptr not monotone");
    nnzC = rp[n];
    if (nnzC > 0 && (!ci || !cv)) fail(HALLAR_EINVAL, "C_col / C_val NULL");
  }
  std::vector<double> diag(n, 0.0);
  // per-row sorted, duplicate-summed off-diagonal entries of C
  std::vector<int64_t> crp(n + 1, 0);
  std::vector<int32_t> ccol;
  std::vector<double> cval;
  ccol.reserve(nnzC);
  cval.reserve(nnzC);
  {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = 0; i < n; ++i) {
      row.clear();
      const int64_t e0 = rp ? rp[i] : 0, e1 = rp ? rp[i + 1] : 0;
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t j = ci[e];
        if (j < 0 || j >= n) fail(HALLAR_EINVAL, "C column index out of range");
        if (!std::isfinite(cv[e])) fail(HALLAR_EINVAL, "C has a non-finite value");
        if (j == i) diag[i] += cv[e];
        else row.emplace_back(j, cv[e]);
      }
      std::sort(row.begin(), row.end(),
                [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
                  return x.first < y.first;
                });
      for (size_t k = 0; k < row.size(); ++k) {
        if ((int64_t)ccol.size() > crp[i] && ccol.back() == row[k].first) {
          cval.back() += row[k].second;
        } else {
          ccol.push_back(row[k].first);
          cval.push_back(row[k].second);
        }
      }
      crp[i + 1] = (int64_t)ccol.size();
    }
  }
  // symmetry: every stored (i, j, v) has its (j, i, v)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = crp[i]; e < crp[i + 1]; ++e) {
      const int32_t j = ccol[e];
      auto b0 = ccol.begin() + crp[j], b1 = ccol.begin() + crp[j + 1];
      auto it = std::lower_bound(b0, b1, (int32_t)i);
      if (it == b1 || *it != i) fail(HALLAR_EINVAL, "C is not symmetric (pattern)");
      const double vt = cval[it - ccol.begin()];
      if (std::fabs(vt - cval[e]) > 1e-12 * std::fmax(std::fabs(vt), std::fabs(cval[e])))
        fail(HALLAR_EINVAL, "C is not symmetric (values)");
    }
  const int64_t nnzOff = (int64_t)ccol.size();
  // induced 1-norm of C = C_sparse + C_J 11^T + C_I I: C is symmetric, so
  // column j's absolute sum is row j's: stored off-diagonals |C_ij + C_J|,
  // the diagonal |C_jj + C_J + C_I| and |C_J| for every other entry
  double cn1 = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t e = crp[j]; e < crp[j + 1]; ++e) s += std::fabs(cval[e] + C_J);
    s += std::fabs(diag[j] + C_J + C_I);
    s += std::fabs(C_J) * (double)(n - (crp[j + 1] - crp[j]) - 1);
    cn1 = std::fmax(cn1, s);
  }
  double bn1 = 0.0;
  for (int64_t l = 0; l < m; ++l) bn1 += std::fabs(b[l]);

  P.api_family = family;
  P.n = n;
  P.n1 = family == HALLAR_OBSERVED ? n1 : 0;
  P.m = m;
  P.m_pairs = family == HALLAR_DIAG ? 0 : m_pairs;
  P.has_trace = family == HALLAR_DIAG ? 0 : (has_trace ? 1 : 0);
  P.C_J = C_J;
  P.C_I = C_I;
  P.tau2 = tau2;
  P.b_norm1 = bn1;
  P.c_norm1 = cn1;
  std::vector<double> cdiag(n);
  for (int64_t i = 0; i < n; ++i) cdiag[i] = diag[i] + C_I;

  std::vector<int32_t> rowptr(n + 1, 0), col, code;
  std::vector<double> val;
  if (family == HALLAR_DIAG) {
    P.fam = FAM_DIAG;
    if (nnzOff >= (int64_t)INT32_MAX) fail(HALLAR_EINVAL, "too many nonzeros");
    for (int64_t i = 0; i <= n; ++i) rowptr[i] = (int32_t)crp[i];
    col = ccol;
    val = cval;
  } else {
    P.fam = nnzOff > 0 ? FAM_EDGE_C : FAM_EDGE;
    const int64_t off = family == HALLAR_OBSERVED ? n1 : 0;
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t l = 0; l < m_pairs; ++l) {
      if (family == HALLAR_OBSERVED) {
        if (pi[l] < 0 || pi[l] >= n1 || pj[l] < 0 || pj[l] >= n - n1)
          fail(HALLAR_EINVAL, "observed pair index out of range");
      } else {
        if (pi[l] < 0 || pi[l] >= n || pj[l] < 0 || pj[l] >= n)
          fail(HALLAR_EINVAL, "pair index out of range");
        if (pi[l] == pj[l]) fail(HALLAR_EINVAL, "pair with i == j");
      }
      cnt[pi[l] + 1]++;
      cnt[pj[l] + off + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += crp[i + 1] - crp[i];
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    const int64_t tot = cnt[n];
    if (tot >= (int64_t)INT32_MAX) fail(HALLAR_EINVAL, "too many nonzeros");
    col.assign(tot, 0);
    code.assign(tot, 0);
    if (nnzOff > 0) val.assign(tot, 0.0);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t l = 0; l < m_pairs; ++l) {
      const int64_t a = pi[l], bb = (int64_t)pj[l] + off;
      int64_t e = pos[a]++;
      col[e] = (int32_t)bb;
      code[e] = (int32_t)l;                // owner
      e = pos[bb]++;
      col[e] = (int32_t)a;
      code[e] = (int32_t)(-l - 1);         // mirror
    }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e2 = crp[i]; e2 < crp[i + 1]; ++e2) {
        const int64_t e = pos[i]++;
        col[e] = ccol[e2];
        code[e] = kNoCons;
        val[e] = cval[e2];
      }
    for (int64_t i = 0; i <= n; ++i) rowptr[i] = (int32_t)cnt[i];
  }
  P.nnz = (int64_t)col.size();
  P.rowptr = std::move(rowptr);
  P.col = std::move(col);
  P.code = std::move(code);
  P.val = std::move(val);
  P.cdiag = std::move(cdiag);
  P.b.assign(b, b + m);
}

namespace {

// device copies of a merged problem (float copies too for the mixed form)
void upload_problem(Ctx* c, const HostProblem& H) {
  Problem& P = c->P;
  P.fam = H.fam;
  P.api_family = H.api_family;
  P.n = H.n;
  P.n1 = H.n1;
  P.m = H.m;
  P.m_pairs = H.m_pairs;
  P.nnz = H.nnz;
  P.has_trace = H.has_trace;
  P.C_J = H.C_J;
  P.C_I = H.C_I;
  P.tau2 = H.tau2;
  P.b_norm1 = H.b_norm1;
  P.c_norm1 = H.c_norm1;
  P.rowptr = upload(c, H.rowptr.data(), H.rowptr.size());
  P.col = upload(c, H.col.data(), H.col.size());
  if (!H.code.empty()) P.code = upload(c, H.code.data(), H.code.size());
  if (!H.val.empty()) {
    P.cval = upload(c, H.val.data(), H.val.size());
    std::vector<float> v32(H.val.begin(), H.val.end());
    P.cval32 = upload(c, v32.data(), v32.size());
  }
  P.cdiag = upload(c, H.cdiag.data(), H.cdiag.size());
  P.b = upload(c, H.b.data(), H.b.size());
  if (c->opt.precision == HALLAR_MIXED) {
    std::vector<float> cd32(H.cdiag.begin(), H.cdiag.end()), b32(H.b.begin(), H.b.end());
    P.cdiag32 = upload(c, cd32.data(), cd32.size());
    P.b32 = upload(c, b32.data(), b32.size());
  }
}

// factor input: a device pointer to n x ld (padded) data
const void* stage_factor(Ctx* c, const void* U, int r, int ld) {
  const size_t es = elem_size(c);
  const int64_t n = c->P.n;
  const bool dev = is_device_ptr(U);
  if (dev && r == ld && ((uintptr_t)U % 16) == 0) return U;
  const void* src = U;
  if (!dev) {
    void* raw = ensure_buffer(c, &c->stage_w, &c->stage_w_bytes, (size_t)n * r * es);
    HL_CUDA(cudaMemcpyAsync(raw, U, (size_t)n * r * es, cudaMemcpyHostToDevice, c->stream));
    if (r == ld) return raw;
    src = raw;
  }
  void* dst = ensure_buffer(c, &c->stage_u, &c->stage_u_bytes, (size_t)n * ld * es);
  launch_pad_copy(c, src, r, dst, ld, r, 1.0);
  return dst;
}

const double* stage_dvec(Ctx* c, const double* v, int64_t len, double** buf, size_t* bytes) {
  if (!v) return nullptr;
  if (is_device_ptr(v)) return v;
  double* d = (double*)ensure_buffer(c, (void**)buf, bytes, (size_t)len * sizeof(double));
  HL_CUDA(cudaMemcpyAsync(d, v, len * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return d;
}

// copy an n x ld device factor to a user n x r array (host or device)
void unstage_factor(Ctx* c, const void* src, int ld, void* dst, int r) {
  const size_t es = elem_size(c);
  const int64_t n = c->P.n;
  const bool dev = is_device_ptr(dst);
  const void* packed = src;
  if (r != ld) {
    void* tmpb = ensure_buffer(c, &c->stage_wout, &c->stage_wout_bytes, (size_t)n * r * es);
    launch_pad_copy(c, src, ld, tmpb, r, r, 1.0);
    packed = tmpb;
  }
  HL_CUDA(cudaMemcpyAsync(dst, packed, (size_t)n * r * es,
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
}

void copy_out_dvec(Ctx* c, double* dst, const double* src, int64_t len) {
  HL_CUDA(cudaMemcpyAsync(dst, src, len * sizeof(double),
                          is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream));
}

template <class F>
hallar_status guarded(Ctx* c, F&& f) {
  if (!c) return HALLAR_EINVAL;
  try {
    HL_CUDA(cudaSetDevice(c->device));
    c->last_error.clear();
    return f();
  } catch (const Err& e) {
    c->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    c->last_error = "host allocation failed";
    return HALLAR_ENOMEM;
  } catch (...) {
    c->last_error = "unexpected exception";
    return HALLAR_ECUDA;
  }
}

void release(Ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  for (void* p : c->owned) cudaFreeAsync(p, c->stream);
  c->owned.clear();
  if (c->stream) cudaStreamSynchronize(c->stream);
  pinned_scalars_release(c->h_scal);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace
}  // namespace hallar

using namespace hallar;

extern "C" {

hallar_status hallar_default_options(hallar_options* o) {
  if (!o) return HALLAR_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-5;
  o->sigma = 0.3;
  o->chi = 0.5;
  o->lambda0 = 1.0;
  o->beta0 = 1.0;
  o->beta_max = 1e8;
  o->eps_decay = 0.5;
  o->eps1_rel = 1e-2;
  o->lanczos_tol_rel = 0.5;
  o->time_limit_s = 3600.0;
  o->lambda_kappa = 0.0;
  o->r_cap = 32;
  o->max_outer = 300;
  o->max_hlr = 100;
  o->max_aipp = 20000;
  o->max_fista = 400;
  o->lanczos_kmax = 300;
  o->precision = HALLAR_FP64;
  o->verbose = 0;
  o->promote = 1;
  o->seed = 0;
  o->stream = nullptr;
  return HALLAR_OK;
}

hallar_status hallar_create(int64_t n, int64_t n1, const int64_t* C_rowptr, const int32_t* C_col,
                            const double* C_val, double C_J, double C_I, int32_t family,
                            int64_t m_pairs, const int32_t* cons_i, const int32_t* cons_j,
                            int32_t has_trace_row, const double* b, double tau2,
                            const hallar_options* opt, hallar_t* out) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out is NULL";
    return HALLAR_EINVAL;
  }
  *out = nullptr;
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return HALLAR_ENOMEM;
  try {
    if (opt) c->opt = *opt;
    else hallar_default_options(&c->opt);
    const hallar_options& o = c->opt;
    if (o.precision != HALLAR_FP64 && o.precision != HALLAR_MIXED)
      fail(HALLAR_EINVAL, "unknown precision");
    if (o.r_cap < 1 || o.r_cap > 89) fail(HALLAR_EINVAL, "r_cap must be in [1, 89]");
    if (!(o.tol > 0.0) || !(o.chi > 0.0 && o.chi < 1.0) || !(o.sigma > 0.0) ||
        !(o.lambda0 > 0.0) || !(o.beta0 > 0.0) || !(o.beta_max >= o.beta0) ||
        !(o.eps_decay > 0.0 && o.eps_decay <= 1.0) || !(o.eps1_rel > 0.0) ||
        !(o.lanczos_tol_rel > 0.0) || !(o.time_limit_s > 0.0) || o.max_fista < 1 ||
        o.max_aipp < 1 || o.max_outer < 1 || o.max_hlr < 1 || o.lanczos_kmax < 2 ||
        (o.promote != 0 && o.promote != 1) || !(o.lambda_kappa >= 0.0) ||
        !std::isfinite(o.lambda_kappa))
      fail(HALLAR_EINVAL, "invalid options");
    HL_CUDA(cudaGetDevice(&c->device));
    HL_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    if (o.stream) {
      c->stream = (cudaStream_t)o.stream;
    } else {
      HL_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    // partial rows: kMaxRed scalars per block for grid reductions, or the
    // 2 (ld + 1) column sums per block of the pre-pass (ld <= kColsumMax)
    c->red.partials = dalloc<double>(c, (size_t)kMaxBlocks * (2 * kColsumMax + 2));
    c->red.counter = dalloc<unsigned>(c, 16);
    HL_CUDA(cudaMemsetAsync(c->red.counter, 0, 16 * sizeof(unsigned), c->stream));
    c->d_scal = dalloc<double>(c, S_COUNT);
    HL_CUDA(cudaMemsetAsync(c->d_scal, 0, S_COUNT * sizeof(double), c->stream));
    c->h_scal = pinned_scalars_acquire();
    c->d_colsum = dalloc<double>(c, 4 * kColsumMax);
    HL_CUDA(cudaMemsetAsync(c->d_colsum, 0, 4 * kColsumMax * sizeof(double), c->stream));
    HostProblem hp;
    merge_problem(hp, n, n1, C_rowptr, C_col, C_val, C_J, C_I, family, m_pairs, cons_i, cons_j,
                  has_trace_row, b, tau2);
    upload_problem(c, hp);
    HL_CUDA(cudaStreamSynchronize(c->stream));
  } catch (const Err& e) {
    g_create_error = e.msg;
    release(c);
    return e.st;
  } catch (const std::bad_alloc&) {
    g_create_error = "host allocation failed";
    release(c);
    return HALLAR_ENOMEM;
  }
  *out = c;
  return HALLAR_OK;
}

hallar_status hallar_eval_A(hallar_t h, const void* U, int32_t r, double* T) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!U || !T || r < 1 || r > 256) fail(HALLAR_EINVAL, "hallar_eval_A: bad argument");
    const int ld = padded_ld(c, r);
    const int64_t m = c->P.m;
    const void* Ud = stage_factor(c, U, r, ld);
    double* Td = is_device_ptr(T) ? T
                                  : (double*)ensure_buffer(c, (void**)&c->stage_m0,
                                                           &c->stage_m0_bytes,
                                                           (size_t)(m + 1) * sizeof(double));
    if (c->P.C_J != 0.0 || c->P.has_trace) launch_colsum(c, Ud, ld, c->d_colsum, S_PRE);
    // the multipliers do not enter T: b stands in for p with beta = 0
    const void* bk = c->opt.precision == HALLAR_MIXED ? (const void*)c->P.b32 : (const void*)c->P.b;
    launch_grad(c, Ud, ld, r, bk, 0.0, GradOut{nullptr, nullptr, Td});
    fetch_scalars(c, 0, S_COUNT);
    double* hs = c->h_scal + S_SCALE;
    hs[2] = c->h_scal[S_GRAD] + c->P.C_J * c->h_scal[S_PRE + 1];
    HL_CUDA(cudaMemcpyAsync(Td, hs + 2, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (c->P.has_trace) {
      hs[3] = c->h_scal[S_PRE];
      HL_CUDA(cudaMemcpyAsync(Td + m, hs + 3, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    if (Td != T) copy_out_dvec(c, T, Td, m + 1);
    sync(c);
    return HALLAR_OK;
  });
}

hallar_status hallar_grad(hallar_t h, const void* U, int32_t r, const double* p, double beta,
                          void* W, double* g_val, double* resid) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!U || !W || !p || r < 1 || r > 256 || !std::isfinite(beta))
      fail(HALLAR_EINVAL, "hallar_grad: bad argument");
    const bool mixed = c->opt.precision == HALLAR_MIXED;
    const int ld = padded_ld(c, r);
    const int64_t m = c->P.m;
    const void* Ud = stage_factor(c, U, r, ld);
    const double* pd = stage_dvec(c, p, m, &c->stage_m1, &c->stage_m1_bytes);
    // the kernel reads p and writes r in the factor type
    const void* pk = pd;
    void* rk = nullptr;
    double* rd = nullptr;  // double residual on the device
    if (mixed) {
      void* buf = ensure_buffer(c, &c->stage_pk, &c->stage_pk_bytes, 2 * (size_t)m * sizeof(float));
      launch_to_factor_type(c, m, buf, pd);
      pk = buf;
      if (resid) rk = (float*)buf + m;
    }
    if (resid) {
      rd = is_device_ptr(resid) ? resid
                                : (double*)ensure_buffer(c, (void**)&c->stage_m0,
                                                         &c->stage_m0_bytes,
                                                         (size_t)m * sizeof(double));
      if (!mixed) rk = rd;
    }
    const bool w_direct = is_device_ptr(W) && r == ld && ((uintptr_t)W % 16) == 0;
    void* Wd = w_direct ? W
                        : ensure_buffer(c, &c->stage_wout, &c->stage_wout_bytes,
                                        (size_t)c->P.n * ld * elem_size(c));
    if (c->P.C_J != 0.0 || c->P.has_trace) launch_colsum(c, Ud, ld, c->d_colsum, S_PRE);
    launch_grad(c, Ud, ld, r, pk, beta, GradOut{Wd, rk, nullptr});
    if (mixed && resid) launch_to_double(c, m, rd, rk);
    fetch_scalars(c, 0, S_COUNT);
    const double* hsc = c->h_scal;
    const double T0 = hsc[S_GRAD] + c->P.C_J * hsc[S_PRE + 1];
    double pr = hsc[S_GRAD + 1], rr = hsc[S_GRAD + 2];
    if (c->P.has_trace) {
      double pt = 0.0, bt = 0.0;
      HL_CUDA(cudaMemcpyAsync(&pt, pd + (m - 1), sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
      HL_CUDA(cudaMemcpyAsync(&bt, c->P.b + (m - 1), sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
      HL_CUDA(cudaStreamSynchronize(c->stream));
      const double rt = hsc[S_PRE] - bt;
      pr += pt * rt;
      rr += rt * rt;
      if (rd) {
        c->h_scal[S_SCALE + 3] = rt;
        HL_CUDA(cudaMemcpyAsync(rd + (m - 1), c->h_scal + S_SCALE + 3, sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
      }
    }
    if (g_val) *g_val = T0 + pr + 0.5 * beta * rr;
    if (!w_direct) {
      if (r == ld) {
        HL_CUDA(cudaMemcpyAsync(W, Wd, (size_t)c->P.n * r * elem_size(c),
                                is_device_ptr(W) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
      } else {
        // repack n x ld -> n x r through the stage_u buffer (U is no longer needed)
        void* packed = ensure_buffer(c, &c->stage_u, &c->stage_u_bytes,
                                     (size_t)c->P.n * r * elem_size(c));
        launch_pad_copy(c, Wd, ld, packed, r, r, 1.0);
        HL_CUDA(cudaMemcpyAsync(W, packed, (size_t)c->P.n * r * elem_size(c),
                                is_device_ptr(W) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
      }
    }
    if (resid && rd != resid) copy_out_dvec(c, resid, rd, m);
    sync(c);
    return HALLAR_OK;
  });
}

hallar_status hallar_value_change(hallar_t h, const void* X, const void* Y, int32_t r,
                                  const double* p, double beta, const double* rX, double* dg,
                                  double* rY) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!X || !Y || !p || !dg || r < 1 || r > 256 || !std::isfinite(beta))
      fail(HALLAR_EINVAL, "hallar_value_change: bad argument");
    const bool mixed = c->opt.precision == HALLAR_MIXED;
    const int ld = padded_ld(c, r);
    const int64_t n = c->P.n, m = c->P.m;
    const size_t es = elem_size(c);
    // X through the regular staging buffer, Y through a second one
    const void* Xd = stage_factor(c, X, r, ld);
    const void* Yd = Y;
    if (!(is_device_ptr(Y) && r == ld && ((uintptr_t)Y % 16) == 0)) {
      const void* src = Y;
      if (!is_device_ptr(Y)) {
        void* raw = ensure_buffer(c, &c->stage_wout, &c->stage_wout_bytes, (size_t)n * r * es);
        HL_CUDA(cudaMemcpyAsync(raw, Y, (size_t)n * r * es, cudaMemcpyHostToDevice, c->stream));
        src = raw;
      }
      if (r == ld) {
        Yd = src;
      } else {
        void* dst = ensure_buffer(c, &c->stage_y, &c->stage_y_bytes, (size_t)n * ld * es);
        launch_pad_copy(c, src, r, dst, ld, r, 1.0);
        Yd = dst;
      }
    }
    const double* pd = stage_dvec(c, p, m, &c->stage_m1, &c->stage_m1_bytes);
    // r_X: given, or from one pass of the fused operator at X
    double* rxd = (double*)ensure_buffer(c, (void**)&c->stage_m0, &c->stage_m0_bytes,
                                         (size_t)m * sizeof(double));
    // factor-typed copies of p, r_X and the output r_Y (p, r_X and r_Y
    // themselves in FP64)
    void* pk = (void*)pd;
    void* rxk = rxd;
    void* ryk = nullptr;
    if (mixed) {
      void* buf = ensure_buffer(c, &c->stage_pk, &c->stage_pk_bytes, 3 * (size_t)m * sizeof(float));
      pk = buf;
      rxk = (float*)buf + m;
      ryk = (float*)buf + 2 * m;
      launch_to_factor_type(c, m, pk, pd);
    }
    double* ryd = nullptr;
    if (rY) {
      ryd = is_device_ptr(rY) ? rY
                              : (double*)ensure_buffer(c, (void**)&c->stage_vc, &c->stage_vc_bytes,
                                                       (size_t)m * sizeof(double));
      if (!mixed) ryk = ryd;
    }
    if (rX) {
      HL_CUDA(cudaMemcpyAsync(rxd, rX, m * sizeof(double),
                              is_device_ptr(rX) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
      if (mixed) launch_to_factor_type(c, m, rxk, rxd);
    } else {
      if (c->P.C_J != 0.0 || c->P.has_trace) launch_colsum(c, Xd, ld, c->d_colsum, S_PRE);
      launch_grad(c, Xd, ld, r, pk, 0.0, GradOut{nullptr, rxk, nullptr});
      if (c->P.has_trace) {
        HL_CUDA(cudaMemcpyAsync(c->h_scal + S_SCALE + 4, c->P.b + (m - 1), sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        launch_trace_fix(c, rxk, nullptr, c->d_scal + S_PRE, -c->h_scal[S_SCALE + 4]);
      }
      if (mixed) launch_to_double(c, m, rxd, rxk);
    }
    // the pieces of g(Y) - g(X), as the solver forms them
    if (c->P.C_J != 0.0)
      launch_colsum_diff(c, Xd, Yd, ld, c->d_colsum + kColsumMax, c->d_colsum + 2 * kColsumMax);
    launch_value_change(c, Xd, Yd, ld, r, pk, rxk, ryk);
    if (ryk && c->P.has_trace) launch_trace_fix(c, ryk, rxk, c->d_scal + S_DIFF + 3, 0.0);
    if (mixed && ryk) launch_to_double(c, m, ryd, ryk);
    fetch_scalars(c, 0, S_COUNT);
    const double* hs = c->h_scal;
    const double dT0 = hs[S_DIFF] + (c->P.C_J != 0.0 ? c->P.C_J * hs[S_DIFF + 9] : 0.0);
    double pdT = hs[S_DIFF + 1], q = hs[S_DIFF + 2];
    if (c->P.has_trace) {
      double pt = 0.0, rxt = 0.0;
      HL_CUDA(cudaMemcpyAsync(&pt, pd + (m - 1), sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
      HL_CUDA(cudaMemcpyAsync(&rxt, rxd + (m - 1), sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
      HL_CUDA(cudaStreamSynchronize(c->stream));
      const double dt = hs[S_DIFF + 3];
      pdT += pt * dt;
      q += dt * (2.0 * rxt + dt);
    }
    *dg = dT0 + pdT + 0.5 * beta * q;
    if (rY && ryd != rY) copy_out_dvec(c, rY, ryd, m);
    sync(c);
    return HALLAR_OK;
  });
}

hallar_status hallar_trim_rank(hallar_t h, const void* Y, int32_t r, int32_t k, void* Yout,
                               double* eigs) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!Y || !Yout || r < 1 || r > 90 || k < 1 || k > r)
      fail(HALLAR_EINVAL, "hallar_trim_rank: need 1 <= k <= r <= 90 and non-NULL Y, Yout");
    const int ld = padded_ld(c, r);
    const int ldk = padded_ld(c, k);
    const int64_t n = c->P.n;
    const void* Yd = stage_factor(c, Y, r, ld);
    void* out = ensure_buffer(c, &c->stage_y, &c->stage_y_bytes, (size_t)n * ldk * elem_size(c));
    trim_factor(c, Yd, ld, r, k, out, ldk, eigs);
    unstage_factor(c, out, ldk, Yout, k);
    sync(c);
    return HALLAR_OK;
  });
}

hallar_status hallar_maxcut_round(hallar_t h, const void* U, int32_t r, const double* G,
                                  int32_t trials, int8_t* x_best, double* cuts) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (c->P.api_family != HALLAR_DIAG)
      fail(HALLAR_EINVAL, "hallar_maxcut_round: needs a HALLAR_DIAG (Max-Cut) problem");
    if (!U || !G || !cuts || r < 1 || r > 256 || trials < 1)
      fail(HALLAR_EINVAL, "hallar_maxcut_round: bad argument");
    const int ld = padded_ld(c, r);
    const int64_t n = c->P.n;
    const void* Ud = stage_factor(c, U, r, ld);
    const double* Gd = stage_dvec(c, G, (int64_t)trials * r, &c->stage_m1, &c->stage_m1_bytes);
    int8_t* xs = (int8_t*)ensure_buffer(c, &c->stage_x, &c->stage_x_bytes, 2 * (size_t)n);
    int8_t* xcur = xs;
    int8_t* xbest = xs + n;
    double best = -INFINITY;
    for (int t = 0; t < trials; ++t) {
      launch_round_sign(c, Ud, ld, r, Gd + (size_t)t * r, xcur);
      launch_cut(c, xcur, S_SCALE);
      fetch_scalars(c, S_SCALE, 2);
      const double sx = c->h_scal[S_SCALE + 1];
      cuts[t] = -(c->h_scal[S_SCALE] + c->P.C_J * sx * sx);
      if (cuts[t] > best) {
        best = cuts[t];
        std::swap(xcur, xbest);
      }
    }
    if (x_best)
      HL_CUDA(cudaMemcpyAsync(x_best, xbest, (size_t)n,
                              is_device_ptr(x_best) ? cudaMemcpyDeviceToDevice
                                                    : cudaMemcpyDeviceToHost,
                              c->stream));
    sync(c);
    return HALLAR_OK;
  });
}

hallar_status hallar_factor_entries(hallar_t h, const void* U, int32_t r, const int32_t* a,
                                    const int32_t* b, int64_t count, double* out) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!U || !a || !b || !out || r < 1 || r > 256 || count < 0)
      fail(HALLAR_EINVAL, "hallar_factor_entries: bad argument");
    if (count == 0) return HALLAR_OK;
    const int ld = padded_ld(c, r);
    const int64_t n = c->P.n;
    const void* Ud = stage_factor(c, U, r, ld);
    // index pairs and the output on the device
    const size_t pb = (size_t)count * sizeof(int32_t);
    char* buf = (char*)ensure_buffer(c, &c->stage_pairs, &c->stage_pairs_bytes,
                                     2 * pb + (size_t)count * sizeof(double));
    const int32_t* ad = a;
    const int32_t* bd = b;
    if (!is_device_ptr(a) || !is_device_ptr(b)) {
      // host pairs: validated here, then copied
      for (int64_t t = 0; t < count; ++t)
        if (a[t] < 0 || a[t] >= n || b[t] < 0 || b[t] >= n)
          fail(HALLAR_EINVAL, "hallar_factor_entries: index out of range");
      HL_CUDA(cudaMemcpyAsync(buf, a, pb, cudaMemcpyHostToDevice, c->stream));
      HL_CUDA(cudaMemcpyAsync(buf + pb, b, pb, cudaMemcpyHostToDevice, c->stream));
      ad = (const int32_t*)buf;
      bd = (const int32_t*)(buf + pb);
    }
    double* od = is_device_ptr(out) ? out : (double*)(buf + 2 * pb);
    launch_entries(c, Ud, ld, r, ad, bd, count, od);
    if (od != out) copy_out_dvec(c, out, od, count);
    sync(c);
    return HALLAR_OK;
  });
}

hallar_status hallar_min_eig(hallar_t h, const double* pshift, double tol, int32_t kmax,
                             const double* v0, double* lambda_min, double* v, int32_t* iters,
                             double* resid) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!pshift || !lambda_min || !(tol > 0.0) || kmax < 2)
      fail(HALLAR_EINVAL, "hallar_min_eig: bad argument");
    const int64_t n = c->P.n, m = c->P.m;
    const double* pd = stage_dvec(c, pshift, m, &c->stage_m1, &c->stage_m1_bytes);
    double* work = (double*)ensure_buffer(c, &c->eig_stage, &c->eig_stage_bytes,
                                          2 * (size_t)n * sizeof(double));
    double* v0d = work;
    double* vd = work + n;
    if (v0) {
      HL_CUDA(cudaMemcpyAsync(v0d, v0, n * sizeof(double),
                              is_device_ptr(v0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
    } else {
      launch_splitmix(c, c->opt.seed, v0d, 0.0, nullptr);
    }
    const LanczosOut le = lanczos_min_eig(c, pd, v0d, tol, kmax, 50, vd);
    *lambda_min = le.lambda;
    if (iters) *iters = le.iters;
    if (resid) *resid = le.resid;
    if (v) copy_out_dvec(c, v, vd, n);
    sync(c);
    return le.converged ? HALLAR_OK : HALLAR_ENOTCONV;
  });
}

hallar_status hallar_solve(hallar_t h, const void* U0, int32_t r0, const double* p0,
                           hallar_result* res) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!U0 || r0 < 1 || r0 > c->opt.r_cap) fail(HALLAR_EINVAL, "hallar_solve: bad U0 / r0");
    const int64_t m = c->P.m;
    const size_t es = elem_size(c);
    const void* Ud = U0;
    if (!is_device_ptr(U0)) {
      void* raw = ensure_buffer(c, &c->stage_w, &c->stage_w_bytes, (size_t)c->P.n * r0 * es);
      HL_CUDA(cudaMemcpyAsync(raw, U0, (size_t)c->P.n * r0 * es, cudaMemcpyHostToDevice,
                              c->stream));
      Ud = raw;
    }
    const double* pd = p0 ? stage_dvec(c, p0, m, &c->stage_p0, &c->stage_p0_bytes) : nullptr;
    hallar_result local{};
    return solve(c, Ud, r0, pd, res ? res : &local);
  });
}

hallar_status hallar_get_solution(hallar_t h, void* U, int32_t r_capacity, double* p,
                                  int32_t* rank) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (!c->sol_U) fail(HALLAR_EINVAL, "no solution: call hallar_solve first");
    if (rank) *rank = c->sol_rank;
    if (U) {
      if (r_capacity < c->sol_rank) fail(HALLAR_EINVAL, "r_capacity below the solution rank");
      unstage_factor(c, c->sol_U, c->sol_ld, U, c->sol_rank);
    }
    if (p) copy_out_dvec(c, p, c->sol_p, c->P.m);
    sync(c);
    return HALLAR_OK;
  });
}

hallar_status hallar_profile(hallar_t h, int32_t op, double* ms, int64_t* launches,
                             double* bytes, double* bytes_padded) {
  return guarded(h, [&]() -> hallar_status {
    Ctx* c = h;
    if (op < 0 || op > 2) fail(HALLAR_EINVAL, "hallar_profile: op must be 0, 1 or 2");
    sync(c);
    if (ms)
      for (int k = 0; k < 3; ++k) ms[k] = c->prof_ms[k];
    if (launches)
      for (int k = 0; k < 3; ++k) launches[k] = c->prof_n[k];
    if (bytes)
      for (int k = 0; k < 3; ++k) bytes[k] = c->prof_bytes[k];
    if (bytes_padded)
      for (int k = 0; k < 3; ++k) bytes_padded[k] = c->prof_bytes_pad[k];
    if (op == 1) {
      for (int k = 0; k < 3; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
        c->prof_bytes[k] = 0.0;
        c->prof_bytes_pad[k] = 0.0;
        c->prof_seen[k] = 0;
      }
      c->prof_on = true;
    } else if (op == 2) {
      c->prof_on = false;
    }
    return HALLAR_OK;
  });
}

hallar_status hallar_profile_sampling(hallar_t h, int32_t every) {
  return guarded(h, [&]() -> hallar_status {
    if (every < 1) fail(HALLAR_EINVAL, "hallar_profile_sampling: every must be >= 1");
    h->prof_every = every;
    return HALLAR_OK;
  });
}

hallar_status hallar_get_sizes(hallar_t h, int64_t* n, int64_t* m, int64_t* nnz,
                               int32_t* precision) {
  if (!h) return HALLAR_EINVAL;
  if (n) *n = h->P.n;
  if (m) *m = h->P.m;
  if (nnz) *nnz = h->P.nnz;
  if (precision) *precision = h->opt.precision;
  return HALLAR_OK;
}

hallar_status hallar_check_problem(int64_t n, int64_t n1, const int64_t* C_rowptr,
                                   const int32_t* C_col, const double* C_val, double C_J,
                                   double C_I, int32_t family, int64_t m_pairs,
                                   const int32_t* cons_i, const int32_t* cons_j,
                                   int32_t has_trace_row, const double* b, double tau2,
                                   int64_t* m, int64_t* nnz_merged, double* c_norm1) {
  g_create_error.clear();
  try {
    HostProblem hp;
    merge_problem(hp, n, n1, C_rowptr, C_col, C_val, C_J, C_I, family, m_pairs, cons_i,
                  cons_j, has_trace_row, b, tau2);
    if (m) *m = hp.m;
    if (nnz_merged) *nnz_merged = hp.nnz;
    if (c_norm1) *c_norm1 = hp.c_norm1;
    return HALLAR_OK;
  } catch (const Err& e) {
    g_create_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    g_create_error = "host allocation failed";
    return HALLAR_ENOMEM;
  }
}

hallar_status hallar_merge_general(int64_t n, int64_t m, int64_t count, const int32_t* ell,
                                   const int32_t* ii, const int32_t* jj, const double* val,
                                   int64_t* nnz_S, int64_t* nnz_L, int64_t* rowptr,
                                   int32_t* col, int64_t* lptr, int32_t* lidx, double* lval) {
  g_create_error.clear();
  try {
    if (n <= 0 || n > INT32_MAX || m < 0 || m > INT32_MAX - 1 || count < 0)
      fail(HALLAR_EINVAL, "need 0 < n < 2^31, 0 <= m < 2^31 - 1, count >= 0");
    if (count > 0 && (!ell || !ii || !jj || !val)) fail(HALLAR_EINVAL, "entry arrays are NULL");
    struct Ent {
      int32_t i, j, l;
      double v;
    };
    std::vector<Ent> es;
    es.reserve((size_t)count * 2);
    for (int64_t k = 0; k < count; ++k) {
      const int32_t l = ell[k], i = ii[k], j = jj[k];
      const double v = val[k];
      if (l < 0 || l > m) fail(HALLAR_EINVAL, "entry " + std::to_string(k) + ": matrix index outside 0..m");
      if (i < 0 || j >= n || i > j)
        fail(HALLAR_EINVAL, "entry " + std::to_string(k) + ": need 0 <= i <= j < n (upper triangle)");
      if (!std::isfinite(v)) fail(HALLAR_EINVAL, "entry " + std::to_string(k) + ": non-finite value");
      if (v == 0.0) continue;
      es.push_back({i, j, l, v});
      if (i != j) es.push_back({j, i, l, v});
    }
    std::sort(es.begin(), es.end(), [](const Ent& a, const Ent& b) {
      if (a.i != b.i) return a.i < b.i;
      if (a.j != b.j) return a.j < b.j;
      return a.l < b.l;
    });
    // sum repeats of one (i, j, l) in order, drop exact zeros
    std::vector<Ent> mg;
    mg.reserve(es.size());
    for (size_t k = 0; k < es.size();) {
      Ent e = es[k];
      size_t q = k + 1;
      while (q < es.size() && es[q].i == e.i && es[q].j == e.j && es[q].l == e.l) e.v += es[q++].v;
      if (e.v != 0.0) mg.push_back(e);
      k = q;
    }
    int64_t s = 0;
    for (size_t k = 0; k < mg.size(); ++k)
      if (k == 0 || mg[k].i != mg[k - 1].i || mg[k].j != mg[k - 1].j) ++s;
    if (nnz_S) *nnz_S = s;
    if (nnz_L) *nnz_L = (int64_t)mg.size();
    if (rowptr || col || lptr || lidx || lval) {
      if (!rowptr || !col || !lptr || !lidx || !lval)
        fail(HALLAR_EINVAL, "the output arrays are all NULL (sizes) or all given");
      std::fill(rowptr, rowptr + n + 1, (int64_t)0);
      int64_t e = -1;
      for (size_t k = 0; k < mg.size(); ++k) {
        if (k == 0 || mg[k].i != mg[k - 1].i || mg[k].j != mg[k - 1].j) {
          ++e;
          col[e] = mg[k].j;
          lptr[e] = (int64_t)k;
          rowptr[mg[k].i + 1]++;
        }
        lidx[k] = mg[k].l;
        lval[k] = mg[k].v;
      }
      lptr[s] = (int64_t)mg.size();
      for (int64_t r = 0; r < n; ++r) rowptr[r + 1] += rowptr[r];
    }
    return HALLAR_OK;
  } catch (const Err& e) {
    g_create_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    g_create_error = "host allocation failed";
    return HALLAR_ENOMEM;
  }
}

void hallar_destroy(hallar_t h) { release(h); }

const char* hallar_last_error(hallar_t h) {
  if (!h) return g_create_error.c_str();
  return h->last_error.c_str();
}

const char* hallar_status_string(hallar_status s) {
  switch (s) {
    case HALLAR_OK: return "HALLAR_OK";
    case HALLAR_EINVAL: return "HALLAR_EINVAL";
    case HALLAR_ENOMEM: return "HALLAR_ENOMEM";
    case HALLAR_ECUDA: return "HALLAR_ECUDA";
    case HALLAR_ENOTCONV: return "HALLAR_ENOTCONV";
    case HALLAR_ETIMEOUT: return "HALLAR_ETIMEOUT";
    case HALLAR_ERANK: return "HALLAR_ERANK";
    case HALLAR_ENUMERIC: return "HALLAR_ENUMERIC";
  }
  return "unknown status";
}

}  // extern "C"
