// Gram matrix Y^T Y of a tall-skinny float factor (n x r, r <= 90) on the
// fifth-generation tensor cores: the dense contraction of the rank trim
// (hallar_options.r_cap; the trim keeps the leading eigenvectors of Y^T Y).
//
// Each CTA (four warps) takes a slice of kGramRows rows.  The slice is
// staged 32 rows at a time into shared memory as the transpose Y^T (M = r
// padded to 128 rows, K = 32 rows of Y), split into TF32 parts
// Y = H + L (H = Y rounded to TF32, L = Y - H rounded to TF32), in the
// K-major no-swizzle canonical layout: 8 x 16-byte core matrices, LBO = 128
// bytes between core matrices along K, SBO = 1024 bytes between 8-row
// groups.  One thread issues tcgen05.mma (kind::tf32, M = N = 128, K = 8
// per instruction) into two FP32 accumulators in tensor memory:
//   P1 = H^T H  (TMEM columns 0..127),  P2 = H^T L  (columns 128..255),
// so Y^T Y = P1 + P2 + P2^T up to the dropped L^T L (relative size 2^-22)
// and FP32 accumulation over the slice.  tcgen05.commit arrives on an
// mbarrier that the CTA waits on (an iteration-limited wait: on expiry the
// kernel raises the error flag, frees its tensor memory and returns).  The
// accumulators are read back with tcgen05.ld and written as FP64 partials
// per CTA; a second kernel sums the partials in block order (deterministic).
#include <cstdint>

#include "device_common.cuh"
#include "hallar_internal.cuh"

namespace hallar {

namespace {

constexpr int kGramRows = 1024;       // rows of Y per CTA (one FP32 accumulation)
constexpr int kGramK = 32;            // rows of Y per shared-memory stage
constexpr int kGramM = 128;           // MMA M = N (r padded)
constexpr int kGramThreads = 128;
constexpr int kTileBytes = kGramM * kGramK * 4;   // 16 KB per operand tile
constexpr uint32_t kLBO = 128;        // core matrices along K
constexpr uint32_t kSBO = (kGramK / 4) * 128;     // 8-row groups
constexpr int kTmemCols = 256;
// dynamic shared memory per CTA: at most two CTAs fit on an SM, so their
// 2 x 256 tensor-memory columns never exceed the SM's 512
constexpr int kGramSmem = 100 * 1024;
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (m, k) of a K-major M x K tile (no swizzle)
__device__ __forceinline__ uint32_t tile_off(int m, int k) {
  return (uint32_t)(m >> 3) * kSBO + (uint32_t)(k >> 2) * kLBO + (uint32_t)(m & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

// shared-memory matrix descriptor: start >> 4 in [0,14), LBO >> 4 in
// [16,30), SBO >> 4 in [32,46), descriptor version 1 in [46,48), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) |
         ((uint64_t)(kSBO >> 4) << 32) | (1ull << 46);
}

// instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 in [17,23), M >> 4 in [24,29)
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kGramM >> 3) << 17) |
                            ((uint32_t)(kGramM >> 4) << 24);

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

// wait for the mbarrier phase; false if the iteration limit ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 32 FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kGramThreads) k_gram_tc(const float* __restrict__ Y, int ld,
                                                          int r, int64_t n,
                                                          double* __restrict__ part1,
                                                          double* __restrict__ part2,
                                                          int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* tileH = smem;
  unsigned char* tileL = smem + kTileBytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * kTileBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * kTileBytes + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t mbar_a = smem_u32(mbar);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int64_t row0 = (int64_t)blockIdx.x * kGramRows;
  const int64_t row1 = min(row0 + (int64_t)kGramRows, n);
  uint32_t phase = 0;
  bool ok = true;
  int stage = 0;
  for (int64_t k0 = row0; k0 < row1 && ok; k0 += kGramK, ++stage) {
    // stage Y[k0 : k0 + 32, 0 : 128] transposed, as TF32 parts H and L
    for (int idx = tid; idx < kGramM * kGramK; idx += kGramThreads) {
      const int k = idx / kGramM, m = idx % kGramM;
      const int64_t row = k0 + k;
      const float y = (m < r && row < row1) ? Y[row * ld + m] : 0.0f;
      const uint32_t h = to_tf32(y);
      const uint32_t l = to_tf32(y - __uint_as_float(h));
      const uint32_t off = tile_off(m, k);
      *reinterpret_cast<uint32_t*>(tileH + off) = h;
      *reinterpret_cast<uint32_t*>(tileL + off) = l;
    }
    // generic-proxy stores -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      const uint32_t aH = smem_u32(tileH), aL = smem_u32(tileL);
#pragma unroll
      for (int s = 0; s < kGramK / 8; ++s) {
        const uint32_t acc = (stage > 0 || s > 0) ? 1u : 0u;
        const uint64_t dH = smem_desc(aH + (uint32_t)s * 2u * kLBO);
        const uint64_t dL = smem_desc(aL + (uint32_t)s * 2u * kLBO);
        mma_tf32(tmem, dH, dH, acc);               // P1 += H^T H
        mma_tf32(tmem + kGramM, dH, dL, acc);      // P2 += H^T L
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::
                       "r"(mbar_a)
                   : "memory");
    }
    // the tiles are reused only after the MMAs that read them completed;
    // the outcome of the wait is made uniform over the CTA
    const int waited = mbar_wait(mbar_a, phase) ? 1 : 0;
    ok = __syncthreads_and(waited) != 0;
    if (ok) phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  if (!ok) {
    // an MMA may still be writing the accumulators: wait once more (with
    // the same limit) before the tensor memory is freed
    if (tid == 0) {
      atomicExch(err, 1);
      mbar_wait(mbar_a, phase);
    }
    __syncthreads();
  } else {
    // warp w reads TMEM lanes 32w .. 32w + 31 (rows m of P1 and P2)
    const int m = warp * 32 + (tid & 31);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < r; c0 += 32) {
      float v1[32], v2[32];
      tmem_ld32(lane_base + (uint32_t)c0, v1);
      tmem_ld32(lane_base + (uint32_t)(kGramM + c0), v2);
      if (m < r) {
        const size_t base = (size_t)blockIdx.x * r * r + (size_t)m * r;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int c = c0 + i;
          if (c < r) {
            part1[base + c] = (double)v1[i];
            part2[base + c] = (double)v2[i];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols));
}

// G = sum_b P1_b + sum_b P2_b + (sum_b P2_b)^T, blocks summed in order
__global__ void k_gram_tc_sum(const double* __restrict__ part1, const double* __restrict__ part2,
                              int nblocks, int r, double* __restrict__ G) {
  const int rr = r * r;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < rr; j += gridDim.x * blockDim.x) {
    const int a = j / r, b = j % r;
    const int jt = b * r + a;
    double s1 = 0.0, s2 = 0.0, s2t = 0.0;
    for (int q = 0; q < nblocks; ++q) {
      s1 += part1[(size_t)q * rr + j];
      s2 += part2[(size_t)q * rr + j];
      s2t += part2[(size_t)q * rr + jt];
    }
    G[j] = s1 + s2 + s2t;
  }
}

}  // namespace

void launch_gram_tc(Ctx* c, const void* U, int ld, int r, double* G) {
  if (r < 1 || r > 90) fail(HALLAR_EINVAL, "tensor-core Gram supports ranks up to 90");
  const int64_t n = c->P.n;
  const int grid = (int)((n + kGramRows - 1) / kGramRows);
  const size_t pbytes = (size_t)grid * r * r * sizeof(double);
  char* buf = (char*)ensure_buffer(c, &c->gram_part, &c->gram_part_bytes, 2 * pbytes + 64);
  double* part1 = (double*)buf;
  double* part2 = (double*)(buf + pbytes);
  int* err = (int*)(buf + 2 * pbytes);
  static bool attr_set[64] = {};
  if (c->device < 64 && !attr_set[c->device]) {
    HL_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kGramSmem));
    attr_set[c->device] = true;
  }
  HL_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  k_gram_tc<<<grid, kGramThreads, kGramSmem, c->stream>>>((const float*)U, ld, r, n, part1,
                                                          part2, err);
  HL_CHECK_LAUNCH(c);
  k_gram_tc_sum<<<(r * r + 127) / 128, 128, 0, c->stream>>>(part1, part2, grid, r, G);
  HL_CHECK_LAUNCH(c);
  int herr = 0;
  HL_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HL_CUDA(cudaStreamSynchronize(c->stream));
  if (herr) fail(HALLAR_ECUDA, "tensor-core Gram: an mbarrier wait ran out");
}

}  // namespace hallar
