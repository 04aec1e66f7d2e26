// Dense BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the
// proposal network: C[m][n] = sum_k A[m][k] B[n][k] with FP32 accumulation in
// tensor memory (TMEM) and a fused epilogue (bias, GELU, FP32 / BF16 outputs).
//
// Operands are row-major BF16 with K contiguous ("K-major"), zero padded to
// Mp, Np (multiples of 128) and Kp (a multiple of 64), so every TMA box lies
// inside its tensor.  One CTA computes a 128 x BN tile (BN = 128 or 64, the
// narrower one when 128-wide tiles would leave SMs idle) over one K range
// (split K: the ranges' partial sums go to separate slices that a second
// kernel adds up in a fixed order):
//   warp 0, one thread: TMA producer -- 128 x 64 (A) and BN x 64 (B) tiles,
//     128-byte swizzle, into a shared-memory ring of 8 (BN = 64) or 6
//     (BN = 128) stages, ~192 KB (mbarrier with tx count);
//   warp 1, one thread: issues tcgen05.mma (M=128, N=BN, K=16) per 16-wide
//     K slice and commits each stage back to the producer;
//   all 4 warps: read the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31 = tile rows), 32 x 32 blocks at a time, pass each
//     block through shared memory (the ring, free by then) so that a warp
//     writes whole rows, and apply the epilogue on the way out.
// Every mbarrier wait is bounded (about 2 s of wall time); on a timeout the
// kernel records an error flag, still frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "opf_internal.h"

namespace opf {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kBM = 128, kBK = 64;
template <int BN>
__host__ __device__ constexpr int stages() {
  return BN == 64 ? 8 : 6;
}
constexpr int kTileA = kBM * kBK * 2;  // 128 rows x 128 bytes
constexpr unsigned long long kWaitNs = 2000000000ull;
// instruction descriptor (kind::f16): D = F32 (bits 4-5), A = B = BF16 (bits
// 7-9, 10-12), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28)
template <int BN>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}
template <int BN>
constexpr size_t smem_bytes() {
  return 1024 + (size_t)stages<BN>() * (kTileA + BN * kBK * 2) + 256;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait for the phase of the given parity to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > kWaitNs) return false;
    __nanosleep(64);
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: 8-row x 128-byte atoms, 1024 bytes apart (stride offset).
__device__ __forceinline__ unsigned long long sw128_desc(uint32_t saddr) {
  unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
  d |= 1ull << 16;                  // leading offset (unused for swizzled K-major)
  d |= (unsigned long long)(1024 >> 4) << 32;
  d |= 1ull << 46;                  // descriptor version
  d |= 2ull << 61;                  // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, unsigned long long a, unsigned long long b,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int nk_all,
              int nsplit, TcEpilogue e, float* part, int* err) {
  constexpr int kTileB = BN * kBK * 2;
  constexpr int kStages = stages<BN>();
  constexpr uint32_t kCols = BN;  // FP32 accumulator: 128 lanes x BN columns
  static_assert(4 * 32 * 33 * 4 <= kStages * kTileA, "epilogue staging must fit in the A ring");
  extern __shared__ unsigned char sraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sraw + 1023) & ~(uintptr_t)1023);  // 128B swizzle: 1 KB aligned
  unsigned char* sA = sm;
  unsigned char* sB = sm + kStages * kTileA;
  uint64_t* bars = (uint64_t*)(sB + kStages * kTileB);  // full[kStages], empty[kStages], done
  uint32_t* tmem_holder = (uint32_t*)(bars + 2 * kStages + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  // this CTA's range of 64-wide K blocks
  const int z = blockIdx.z, per = (nk_all + nsplit - 1) / nsplit;
  const int kb0 = z * per, nk = max(0, min(nk_all, kb0 + per) - kb0);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + kStages + s); };
  const uint32_t done = smem_u32(bars + 2 * kStages);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // whole warp: allocate the accumulator columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  bool ok = true;

  if (warp == 0 && lane == 0) {  // TMA producer
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages && !mbar_wait(empty(s), ((kb / kStages) - 1) & 1)) {
        ok = false;
        break;
      }
      mbar_expect_tx(full(s), kTileA + kTileB);
      tma_load_2d(smem_u32(sA + s * kTileA), &ta, (kb0 + kb) * kBK, m0, full(s));
      tma_load_2d(smem_u32(sB + s * kTileB), &tb, (kb0 + kb) * kBK, n0, full(s));
      ++issued;
    }
    if (!ok)  // let the copies already issued land before the CTA can exit
      for (int kb = issued - 1; kb >= 0 && kb >= issued - kStages; --kb)
        mbar_wait(full(kb % kStages), (kb / kStages) & 1);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(full(s), (kb / kStages) & 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * kTileA), b0 = smem_u32(sB + s * kTileB);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)  // 16 BF16 = 32 bytes per K slice
        umma_bf16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc<BN>(), (kb | kk) != 0);
      umma_commit(empty(s));
    }
    umma_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();

  // epilogue: TMEM lane = tile row (warp w: rows 32w..32w+31), 32 columns per
  // load; each 32 x 32 block goes through this warp's slice of the A ring
  // (free once every MMA has completed; rows padded to 33 floats, so neither
  // the row-wise writes nor the column-wise reads meet bank conflicts), then
  // lane j takes column n0 + c0 + j of each of the 32 rows: coalesced stores.
  if (!mbar_wait(done, 0)) ok = false;
  tc_fence_after();
  float* stage = (float*)sA + warp * 32 * 33;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = nk ? __uint_as_float(v[j]) : 0.f;
    __syncwarp();
    const int n = n0 + c0 + lane;
    const float bn = (!part && e.bias && n < N) ? e.bias[n] : 0.f;
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const int row = m0 + warp * 32 + rr;
      if (row >= M || n >= N) continue;
      float x = stage[rr * 33 + lane];
      if (part) {  // split K: raw partial sums into this split's slice
        part[((long)z * M + row) * N + n] = x;
      } else {
        x += bn;
        const long o = (long)row * e.ldo + n;
        if (e.pre_f32) e.pre_f32[o] = x;
        if (e.gelu) x = gelu_f(x);
        if (e.out_f32) e.out_f32[o] = e.accumulate ? e.out_f32[o] + x : x;
        if (e.out_bf16) ((bf16*)e.out_bf16)[o] = __float2bfloat16(x);
      }
    }
    __syncwarp();
  }
  if (!ok) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
}

// out[m][n] (row stride ldo) = sum over splits, in split order, of part[z][m][n]
__global__ void k_split_sum(const float* __restrict__ part, int nsplit, int M, int N, float* __restrict__ out,
                            long ldo, int accumulate) {
  const long total = (long)M * N;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nsplit; ++z) s += part[(long)z * total + i];
    const long m = i / N, n = i - m * N;
    float* o = out + m * ldo + n;
    *o = accumulate ? *o + s : s;
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  });
  return fn;
}

// 2-D map of a row-major BF16 matrix [rows][Kp]: boxes of box_rows rows x 64 columns
bool make_map(CUtensorMap* m, const void* base, int rows, int Kp, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
bool set_attr() {
  return cudaFuncSetAttribute(k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<BN>()) ==
         cudaSuccess;
}

}  // namespace

int tc_gemm(const void* A, const void* B, int M, int N, int Mp, int Np, int Kp, const TcEpilogue& e, int* d_err,
            cudaStream_t st, float* work, long work_floats) {
  if (M < 1 || N < 1 || M > Mp || N > Np || Mp % kBM || Np % 128 || Kp < kBK || Kp % kBK ||
      ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) {
    set_last_error("tc_gemm: operand shapes must be padded to 128 x 64 multiples on 16-byte boundaries");
    return OPF_EINVAL;
  }
  static std::once_flag once;
  static bool attr_ok = false;
  std::call_once(once, [] { attr_ok = set_attr<128>() && set_attr<64>(); });
  // launch shape: 64-wide tiles when 128-wide ones leave SMs idle; split K
  // (plain outputs only) while the tiles still fill fewer than 152 SMs
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles128 = (Mp / kBM) * (Np / 128);
  const int BN = tiles128 < sms ? 64 : 128;
  const int tiles = (Mp / kBM) * (Np / BN), nk = Kp / kBK;
  int nsplit = 1;
  const bool plain = !e.bias && !e.gelu && !e.pre_f32 && !e.out_bf16 && e.out_f32;
  if (plain && work)
    while (nsplit < 8 && tiles * nsplit * 2 <= 2 * sms && nk / (nsplit * 2) >= 4 &&
           (long)(nsplit * 2) * M * N <= work_floats)
      nsplit *= 2;
  CUtensorMap ta, tb;
  if (!attr_ok || !make_map(&ta, A, Mp, Kp, kBM) || !make_map(&tb, B, Np, Kp, BN)) {
    set_last_error("tc_gemm: tensor map or kernel attribute setup failed");
    return OPF_ECUDA;
  }
  dim3 grid(Np / BN, Mp / kBM, nsplit);
  float* part = nsplit > 1 ? work : nullptr;
  if (BN == 64)
    k_tc_gemm<64><<<grid, 128, smem_bytes<64>(), st>>>(ta, tb, M, N, nk, nsplit, e, part, d_err);
  else
    k_tc_gemm<128><<<grid, 128, smem_bytes<128>(), st>>>(ta, tb, M, N, nk, nsplit, e, part, d_err);
  if (part) {
    const long total = (long)M * N;
    const int blocks = (int)std::min<long>((total + 255) / 256, 4L * sms);
    k_split_sum<<<blocks, 256, 0, st>>>(part, nsplit, M, N, e.out_f32, e.ldo, e.accumulate);
  }
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_last_error(std::string("tc_gemm launch: ") + cudaGetErrorString(err));
    return OPF_ECUDA;
  }
  return OPF_OK;
}

}  // namespace opf
