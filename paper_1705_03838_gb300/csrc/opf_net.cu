// Proposal network for Newton-Krylov initial guesses: a 1-D convolution net
// over the radial points acting on the lowest Fourier modes of a state.
//
//   h1 = gelu(conv3(x;  W1, b1))          x: [B][L][Cin]   (L radial points)
//   h2 = gelu(conv3(h1; W2, b2))          h: [B][L][H]
//   y  = conv3(h2; W3, b3)                y: [B][L][Cin]   (correction of x)
//   z  = Wh mean_l(h2) + bh               z: [B][2]        (period, shift)
//   loss = mean((y - ty)^2) + lambda mean((z - tz)^2)
//
// conv3 is a width-3 convolution along l with zero padding.  Every
// convolution and its two backward products is one GEMM on BF16 operands
// with FP32 accumulation (mma.sync m16n8k16 tensor-core instructions); the
// im2col matrix is never formed -- the tile loader reads x[b][l + j - 1][c]
// for column j*C + c.  Master weights and Adam moments are FP32.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "opf_internal.h"

namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ GEMM
// C[m][n] = sum_k A(m,k) B(n,k).  Operand addressing modes:
enum AMode { A_ROWMAJOR = 0, A_IM2COL = 1, A_IM2COL_REV = 2, A_COLMAJOR = 3 };
enum BMode { B_ROWMAJOR = 0, B_COLMAJOR = 1, B_WT_SHIFT = 2, B_IM2COL_T = 3 };

struct GemmArgs {
  int M, N, K;
  // A
  const void* A;
  int a_mode, a_f32;  // a_f32: A is float (converted to bf16 on load)
  long lda;           // ROWMAJOR: A[m*lda + k]; COLMAJOR: A[k*lda + m]
  int L, C;           // IM2COL: m = b*L + l, k = j*C + c, src x[(b*L + l + s(j-1))*C + c]
  // B
  const void* Bp;
  int b_mode, b_f32;
  long ldb;           // ROWMAJOR: B[n*ldb + k]; COLMAJOR: B[k*ldb + n]
  int bN, bC;         // WT_SHIFT: k = j*bN + o, value W[o*ldb + j*bC + n]
                      // IM2COL_T: n = j*bC + c, k = b*bN + l -> x[(b*bN + l + j - 1)*bC + c]
  // epilogue
  const float* bias;  // per n (may be null)
  int gelu;           // 1: out = gelu(acc + bias)
  float* out_f32;     // [m][n] (ld = N), may be null
  float* pre_f32;     // pre-activation (acc + bias), may be null
  bf16* out_bf16;     // may be null
  int accumulate;     // out_f32 += acc
};

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

template <typename T>
__device__ __forceinline__ float ldf(const void* p, long i) {
  return (float)((const T*)p)[i];
}

__device__ __forceinline__ float load_a(const GemmArgs& g, int m, int k) {
  if (m >= g.M || k >= g.K) return 0.f;
  long idx;
  switch (g.a_mode) {
    case A_ROWMAJOR: idx = (long)m * g.lda + k; break;
    case A_COLMAJOR: idx = (long)k * g.lda + m; break;
    default: {
      const int b = m / g.L, l = m - b * g.L, j = k / g.C, c = k - j * g.C;
      const int ls = l + (g.a_mode == A_IM2COL ? (j - 1) : (1 - j));
      if (ls < 0 || ls >= g.L) return 0.f;
      idx = ((long)b * g.L + ls) * g.C + c;
    }
  }
  return g.a_f32 ? ldf<float>(g.A, idx) : __bfloat162float(((const bf16*)g.A)[idx]);
}

__device__ __forceinline__ float load_b(const GemmArgs& g, int n, int k) {
  if (n >= g.N || k >= g.K) return 0.f;
  long idx;
  switch (g.b_mode) {
    case B_ROWMAJOR: idx = (long)n * g.ldb + k; break;
    case B_COLMAJOR: idx = (long)k * g.ldb + n; break;
    case B_WT_SHIFT: {
      const int j = k / g.bN, o = k - j * g.bN;
      idx = (long)o * g.ldb + (long)j * g.bC + n;
      break;
    }
    default: {  // B_IM2COL_T
      const int L = g.bN, C = g.bC;
      const int b = k / L, l = k - b * L, j = n / C, c = n - j * C;
      const int ls = l + j - 1;
      if (ls < 0 || ls >= L) return 0.f;
      idx = ((long)b * L + ls) * C + c;
    }
  }
  return g.b_f32 ? ldf<float>(g.Bp, idx) : __bfloat162float(((const bf16*)g.Bp)[idx]);
}

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

__device__ __forceinline__ uint32_t pack2(const bf16* p) { return *(const uint32_t*)p; }

__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
  __shared__ __align__(16) bf16 As[BM][BK + PAD];
  __shared__ __align__(16) bf16 Bs[BN][BK + PAD];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 128) {
      const int r = e / BK, kk = e % BK;
      As[r][kk] = __float2bfloat16(load_a(g, m0 + r, k0 + kk));
      Bs[r][kk] = __float2bfloat16(load_b(g, n0 + r, k0 + kk));
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = wm + a * 16 + gq;
        af[a][0] = pack2(&As[r][ks + tq * 2]);
        af[a][1] = pack2(&As[r + 8][ks + tq * 2]);
        af[a][2] = pack2(&As[r][ks + tq * 2 + 8]);
        af[a][3] = pack2(&As[r + 8][ks + tq * 2 + 8]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = wn + b * 8 + gq;
        bfr[b][0] = pack2(&Bs[c][ks + tq * 2]);
        bfr[b][1] = pack2(&Bs[c][ks + tq * 2 + 8]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
              "{%8,%9}, {%0,%1,%2,%3};"
              : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
              : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bfr[b][0]),
                "r"(bfr[b][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int m = m0 + wm + a * 16 + gq + h * 8;
          const int n = n0 + wn + b * 8 + tq * 2 + e;
          if (m >= g.M || n >= g.N) continue;
          float v = acc[a][b][h * 2 + e] + (g.bias ? g.bias[n] : 0.f);
          const long o = (long)m * g.N + n;
          if (g.pre_f32) g.pre_f32[o] = v;
          if (g.gelu) v = gelu_f(v);
          if (g.out_f32) g.out_f32[o] = g.accumulate ? g.out_f32[o] + v : v;
          if (g.out_bf16) g.out_bf16[o] = __float2bfloat16(v);
        }
}

void gemm(const GemmArgs& g, cudaStream_t st) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  k_gemm<<<grid, 128, 0, st>>>(g);
}

GemmArgs gemm_args(int M, int N, int K) {
  GemmArgs g;
  std::memset(&g, 0, sizeof g);
  g.M = M;
  g.N = N;
  g.K = K;
  return g;
}

// ------------------------------------------------------------------ small kernels
__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// dZ = dY * gelu'(pre), stored as bf16 (operand of the next GEMMs) and f32
__global__ void k_gelu_back(const float* __restrict__ dy, const float* __restrict__ pre, bf16* __restrict__ dz,
                            float* __restrict__ dzf, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float v = dy[i] * gelu_grad(pre[i]);
    dz[i] = __float2bfloat16(v);
    if (dzf) dzf[i] = v;
  }
}

// column sums (bias gradients): out[n] = sum_m x[m][n]
__global__ void k_colsum(const float* __restrict__ x, int M, int N, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += x[(long)m * N + n];
  out[n] = s;
}

// mean over l of h2 (bf16 -> f32): pooled[b][c]
__global__ void k_pool(const bf16* __restrict__ h, int B, int L, int C, float* __restrict__ pooled) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * C) return;
  const int b = i / C, c = i % C;
  float s = 0.f;
  for (int l = 0; l < L; ++l) s += __bfloat162float(h[((long)b * L + l) * C + c]);
  pooled[i] = s / L;
}

// head: z[b][o] = sum_c Wh[o][c] pooled[b][c] + bh[o]; loss terms and gradients
__global__ void k_head(const float* __restrict__ pooled, const float* __restrict__ Wh, const float* __restrict__ bh,
                       int B, int C, int O, float* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * O) return;
  const int b = i / O, o = i % O;
  float s = bh[o];
  for (int c = 0; c < C; ++c) s += Wh[o * C + c] * pooled[b * C + c];
  z[i] = s;
}

// residuals r = pred - target and their squared sums (two partial sums)
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ tgt, long n, float scale,
                      float* __restrict__ grad, double* __restrict__ sum) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float r = pred[i] - tgt[i];
    acc += (double)r * r;
    grad[i] = 2.f * scale * r;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(sum, sh[0]);
}

// head backward: dWh[o][c] = sum_b dz[b][o] pooled[b][c]; dbh; dpooled[b][c]
__global__ void k_head_back(const float* __restrict__ dz, const float* __restrict__ pooled,
                            const float* __restrict__ Wh, int B, int C, int O, float* __restrict__ dWh,
                            float* __restrict__ dbh, float* __restrict__ dpooled) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < O * C) {
    const int o = i / C, c = i % C;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dz[b * O + o] * pooled[b * C + c];
    dWh[i] = s;
  }
  if (i < O) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dz[b * O + i];
    dbh[i] = s;
  }
  if (i < B * C) {
    const int b = i / C, c = i % C;
    float s = 0.f;
    for (int o = 0; o < O; ++o) s += dz[b * O + o] * Wh[o * C + c];
    dpooled[i] = s;
  }
}

// add the pooled-mean gradient to dh2 (broadcast over l, divided by L)
__global__ void k_unpool_add(const float* __restrict__ dpooled, int B, int L, int C, float* __restrict__ dh) {
  const long n = (long)B * L * C;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long b = i / ((long)L * C), c = i % C;
    dh[i] += dpooled[b * C + c] / L;
  }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long n, float lr, float b1, float b2, float c1, float c2,
                       float eps, bf16* __restrict__ wb) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    m1[i] = b1 * m1[i] + (1.f - b1) * g[i];
    m2[i] = b2 * m2[i] + (1.f - b2) * g[i] * g[i];
    w[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + eps);
    if (wb) wb[i] = __float2bfloat16(w[i]);
  }
}

int gs(long n) { return (int)std::min<long>((n + 255) / 256, 4096); }

}  // namespace

// ====================================================================== net object
struct opf_net {
  int Cin, H, L, O;
  // parameters (f32 master) in one block: W1 b1 W2 b2 W3 b3 Wh bh
  long off[8], count[8], total;
  float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;
  bf16* Pb = nullptr;  // bf16 copies of the weight matrices (same offsets)
  long step = 0;
  int Bcap = 0;
  // activations / workspace for batch capacity Bcap
  bf16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *dz = nullptr, *dz2 = nullptr;
  float *pre1 = nullptr, *pre2 = nullptr, *y = nullptr, *dy = nullptr, *dh = nullptr;
  float *pooled = nullptr, *z = nullptr, *dzh = nullptr, *dpooled = nullptr;
  double* sums = nullptr;
  cudaStream_t st = nullptr;
};

namespace {
int nfail(const std::string& m) {
  opf::set_last_error(m);
  return OPF_ECUDA;
}
#define NCU(call)                                                                    \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return nfail(std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int net_reserve(opf_net* n, int B) {
  if (B <= n->Bcap) return OPF_OK;
  auto fr = [](void* p) {
    if (p) cudaFree(p);
  };
  fr(n->xb), fr(n->h1), fr(n->h2), fr(n->dz), fr(n->dz2), fr(n->pre1), fr(n->pre2), fr(n->y);
  fr(n->dy), fr(n->dh), fr(n->pooled), fr(n->z), fr(n->dzh), fr(n->dpooled), fr(n->sums);
  const long BL = (long)B * n->L, W = std::max(n->H, n->Cin);
  NCU(cudaMalloc(&n->xb, BL * n->Cin * sizeof(bf16)));
  NCU(cudaMalloc(&n->h1, BL * n->H * sizeof(bf16)));
  NCU(cudaMalloc(&n->h2, BL * n->H * sizeof(bf16)));
  NCU(cudaMalloc(&n->dz, BL * W * sizeof(bf16)));
  NCU(cudaMalloc(&n->dz2, BL * W * sizeof(bf16)));
  NCU(cudaMalloc(&n->pre1, BL * n->H * sizeof(float)));
  NCU(cudaMalloc(&n->pre2, BL * n->H * sizeof(float)));
  NCU(cudaMalloc(&n->y, BL * n->Cin * sizeof(float)));
  NCU(cudaMalloc(&n->dy, BL * W * sizeof(float)));
  NCU(cudaMalloc(&n->dh, BL * W * sizeof(float)));
  NCU(cudaMalloc(&n->pooled, (long)B * n->H * sizeof(float)));
  NCU(cudaMalloc(&n->z, (long)B * n->O * sizeof(float)));
  NCU(cudaMalloc(&n->dzh, (long)B * n->O * sizeof(float)));
  NCU(cudaMalloc(&n->dpooled, (long)B * n->H * sizeof(float)));
  NCU(cudaMalloc(&n->sums, 2 * sizeof(double)));
  n->Bcap = B;
  return OPF_OK;
}

float* Pf(opf_net* n, int i) { return n->P + n->off[i]; }
float* Gf(opf_net* n, int i) { return n->G + n->off[i]; }
bf16* Pbf(opf_net* n, int i) { return n->Pb + n->off[i]; }

// forward for B samples whose features are at x (f32 [B][L][Cin])
int net_forward(opf_net* n, const float* x, int B) {
  const int L = n->L, Ci = n->Cin, H = n->H, O = n->O;
  const long BL = (long)B * L;
  k_to_bf16<<<gs(BL * Ci), 256, 0, n->st>>>(x, n->xb, BL * Ci);
  GemmArgs g = gemm_args((int)BL, H, 3 * Ci);  // layer 1
  g.A = n->xb, g.a_mode = A_IM2COL, g.L = L, g.C = Ci;
  g.Bp = Pbf(n, 0), g.b_mode = B_ROWMAJOR, g.ldb = 3 * Ci;
  g.bias = Pf(n, 1), g.gelu = 1, g.pre_f32 = n->pre1, g.out_bf16 = n->h1;
  gemm(g, n->st);
  g = gemm_args((int)BL, H, 3 * H);  // layer 2
  g.A = n->h1, g.a_mode = A_IM2COL, g.L = L, g.C = H;
  g.Bp = Pbf(n, 2), g.b_mode = B_ROWMAJOR, g.ldb = 3 * H;
  g.bias = Pf(n, 3), g.gelu = 1, g.pre_f32 = n->pre2, g.out_bf16 = n->h2;
  gemm(g, n->st);
  g = gemm_args((int)BL, Ci, 3 * H);  // layer 3 (linear)
  g.A = n->h2, g.a_mode = A_IM2COL, g.L = L, g.C = H;
  g.Bp = Pbf(n, 4), g.b_mode = B_ROWMAJOR, g.ldb = 3 * H;
  g.bias = Pf(n, 5), g.out_f32 = n->y;
  gemm(g, n->st);
  k_pool<<<(B * H + 255) / 256, 256, 0, n->st>>>(n->h2, B, L, H, n->pooled);
  k_head<<<(B * O + 255) / 256, 256, 0, n->st>>>(n->pooled, Pf(n, 6), Pf(n, 7), B, H, O, n->z);
  return OPF_OK;
}

// gradient of one width-3 conv layer given dZ (bf16 [BL][Cout], f32 copy dZf):
//   dW[o][j*Cin + c] = sum_m dZ[m][o] xcol[m][j*Cin + c]     (reduction over m)
//   db[o] = sum_m dZ[m][o]
//   dx[(b,l)][c] = sum_{j,o} dZ[(b, l + 1 - j)][o] W[o][j*Cin + c]
void conv_backward(opf_net* n, int B, const bf16* x, int Cin, int Cout, const bf16* dZ, const float* dZf,
                   const bf16* Wb, float* dW, float* db, float* dx) {
  const int L = n->L;
  const long BL = (long)B * L;
  GemmArgs w = gemm_args(Cout, 3 * Cin, (int)BL);
  w.A = dZ, w.a_mode = A_COLMAJOR, w.lda = Cout;
  w.Bp = x, w.b_mode = B_IM2COL_T, w.bN = L, w.bC = Cin;
  w.out_f32 = dW;
  gemm(w, n->st);
  k_colsum<<<(Cout + 255) / 256, 256, 0, n->st>>>(dZf, (int)BL, Cout, db);
  if (dx) {
    GemmArgs v = gemm_args((int)BL, Cin, 3 * Cout);
    v.A = dZ, v.a_mode = A_IM2COL_REV, v.L = L, v.C = Cout;
    v.Bp = Wb, v.b_mode = B_WT_SHIFT, v.ldb = 3 * Cin, v.bN = Cout, v.bC = Cin;
    v.out_f32 = dx;
    gemm(v, n->st);
  }
}

// loss and all parameter gradients into n->G for targets ty [B][L][Cin], tz [B][O]
int net_gradients(opf_net* n, const float* x, const float* ty, const float* tz, int B, float lambda,
                  double* loss) {
  const int L = n->L, Ci = n->Cin, H = n->H, O = n->O;
  const long BL = (long)B * L;
  int rc = net_forward(n, x, B);
  if (rc) return rc;
  NCU(cudaMemsetAsync(n->sums, 0, 2 * sizeof(double), n->st));
  // dL/dy = 2 (y - ty) / (BL Ci); dL/dz = 2 lambda (z - tz) / (B O)
  k_mse<<<gs(BL * Ci), 256, 0, n->st>>>(n->y, ty, BL * Ci, 1.f / (float)(BL * Ci), n->dy, n->sums);
  k_mse<<<1, 256, 0, n->st>>>(n->z, tz, (long)B * O, lambda / (float)(B * O), n->dzh, n->sums + 1);
  // layer 3 (linear): dZ3 = dy
  k_to_bf16<<<gs(BL * Ci), 256, 0, n->st>>>(n->dy, n->dz, BL * Ci);
  conv_backward(n, B, n->h2, H, Ci, n->dz, n->dy, Pbf(n, 4), Gf(n, 4), Gf(n, 5), n->dh);
  // head: pooled mean of h2
  const int hb = (int)std::max<long>((long)O * H, (long)B * H);
  k_head_back<<<(hb + 255) / 256, 256, 0, n->st>>>(n->dzh, n->pooled, Pf(n, 6), B, H, O, Gf(n, 6), Gf(n, 7),
                                                   n->dpooled);
  k_unpool_add<<<gs(BL * H), 256, 0, n->st>>>(n->dpooled, B, L, H, n->dh);
  // layer 2
  k_gelu_back<<<gs(BL * H), 256, 0, n->st>>>(n->dh, n->pre2, n->dz, n->dy, BL * H);
  conv_backward(n, B, n->h1, H, H, n->dz, n->dy, Pbf(n, 2), Gf(n, 2), Gf(n, 3), n->dh);
  // layer 1 (input gradient not needed)
  k_gelu_back<<<gs(BL * H), 256, 0, n->st>>>(n->dh, n->pre1, n->dz2, n->dy, BL * H);
  conv_backward(n, B, n->xb, Ci, H, n->dz2, n->dy, Pbf(n, 0), Gf(n, 0), Gf(n, 1), nullptr);
  if (loss) {
    double h[2];
    NCU(cudaMemcpyAsync(h, n->sums, sizeof h, cudaMemcpyDeviceToHost, n->st));
    NCU(cudaStreamSynchronize(n->st));
    *loss = h[0] / (double)(BL * Ci) + lambda * h[1] / (double)(B * O);
  }
  NCU(cudaGetLastError());
  return OPF_OK;
}

void refresh_bf16(opf_net* n) {
  k_to_bf16<<<gs(n->total), 256, 0, n->st>>>(n->P, n->Pb, n->total);
}

}  // namespace

extern "C" {

opf_net_t* opf_net_create(int cin, int hidden, int L, int nout, unsigned long long seed) {
  if (cin < 1 || hidden < 1 || L < 1 || nout < 1) {
    opf::set_last_error("opf_net_create: sizes must be positive");
    return nullptr;
  }
  opf_net* n = new opf_net();
  n->Cin = cin;
  n->H = hidden;
  n->L = L;
  n->O = nout;
  const long cnt[8] = {(long)hidden * 3 * cin, hidden, (long)hidden * 3 * hidden, hidden,
                       (long)cin * 3 * hidden, cin, (long)nout * hidden, nout};
  long t = 0;
  for (int i = 0; i < 8; ++i) {
    n->off[i] = t;
    n->count[i] = cnt[i];
    t += (cnt[i] + 63) / 64 * 64;
  }
  n->total = t;
  // deterministic init: uniform(-a, a), a = 1/sqrt(fan_in), biases 0
  std::vector<float> h(t, 0.f);
  unsigned long long z = seed;
  auto next = [&]() {
    z += 0x9E3779B97F4A7C15ull;
    unsigned long long q = z;
    q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ull;
    q = (q ^ (q >> 27)) * 0x94D049BB133111EBull;
    q ^= q >> 31;
    return (double)(q >> 11) * (1.0 / 9007199254740992.0);
  };
  const long fan[8] = {3L * cin, 0, 3L * hidden, 0, 3L * hidden, 0, hidden, 0};
  for (int i = 0; i < 8; i += 2) {
    const double a = 1.0 / std::sqrt((double)fan[i]);
    for (long j = 0; j < cnt[i]; ++j) h[n->off[i] + j] = (float)((2.0 * next() - 1.0) * a);
  }
  if (cudaStreamCreateWithFlags(&n->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&n->P, t * sizeof(float)) != cudaSuccess || cudaMalloc(&n->G, t * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->M1, t * sizeof(float)) != cudaSuccess || cudaMalloc(&n->M2, t * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->Pb, t * sizeof(bf16)) != cudaSuccess) {
    opf::set_last_error("opf_net_create: device allocation failed");
    opf_net_destroy(n);
    return nullptr;
  }
  cudaMemcpy(n->P, h.data(), t * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(n->G, 0, t * sizeof(float));
  cudaMemset(n->M1, 0, t * sizeof(float));
  cudaMemset(n->M2, 0, t * sizeof(float));
  refresh_bf16(n);
  if (cudaStreamSynchronize(n->st) != cudaSuccess) {
    opf::set_last_error("opf_net_create: initialisation failed");
    opf_net_destroy(n);
    return nullptr;
  }
  return n;
}

void opf_net_destroy(opf_net_t* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st);
  for (void* p : {(void*)n->P, (void*)n->G, (void*)n->M1, (void*)n->M2, (void*)n->Pb, (void*)n->xb,
                  (void*)n->h1, (void*)n->h2, (void*)n->dz, (void*)n->dz2, (void*)n->pre1, (void*)n->pre2,
                  (void*)n->y, (void*)n->dy, (void*)n->dh, (void*)n->pooled, (void*)n->z, (void*)n->dzh,
                  (void*)n->dpooled, (void*)n->sums})
    if (p) cudaFree(p);
  if (n->st) cudaStreamDestroy(n->st);
  delete n;
}

int opf_net_param_count(opf_net_t* n, long* total, long* sizes8) {
  if (!n || !total) return OPF_EINVAL;
  long s = 0;
  for (int i = 0; i < 8; ++i) {
    s += n->count[i];
    if (sizes8) sizes8[i] = n->count[i];
  }
  *total = s;
  return OPF_OK;
}

int opf_net_get_params(opf_net_t* n, float* host, int grads) {
  if (!n || !host) return OPF_EINVAL;
  std::vector<float> h(n->total);
  NCU(cudaMemcpy(h.data(), grads ? n->G : n->P, n->total * sizeof(float), cudaMemcpyDeviceToHost));
  long o = 0;
  for (int i = 0; i < 8; ++i)
    for (long j = 0; j < n->count[i]; ++j) host[o++] = h[n->off[i] + j];
  return OPF_OK;
}

int opf_net_set_params(opf_net_t* n, const float* host) {
  if (!n || !host) return OPF_EINVAL;
  std::vector<float> h(n->total, 0.f);
  long o = 0;
  for (int i = 0; i < 8; ++i)
    for (long j = 0; j < n->count[i]; ++j) h[n->off[i] + j] = host[o++];
  NCU(cudaMemcpy(n->P, h.data(), n->total * sizeof(float), cudaMemcpyHostToDevice));
  refresh_bf16(n);
  NCU(cudaStreamSynchronize(n->st));
  return OPF_OK;
}

int opf_net_forward(opf_net_t* n, const float* d_x, int B, float* d_y, float* d_z) {
  if (!n || !d_x || B < 1) return OPF_EINVAL;
  int rc = net_reserve(n, B);
  if (rc) return rc;
  rc = net_forward(n, d_x, B);
  if (rc) return rc;
  const long BL = (long)B * n->L;
  if (d_y) NCU(cudaMemcpyAsync(d_y, n->y, BL * n->Cin * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
  if (d_z) NCU(cudaMemcpyAsync(d_z, n->z, (long)B * n->O * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
  NCU(cudaStreamSynchronize(n->st));
  NCU(cudaGetLastError());
  return OPF_OK;
}

int opf_net_gradients(opf_net_t* n, const float* d_x, const float* d_ty, const float* d_tz, int B,
                      float lambda, double* loss) {
  if (!n || !d_x || !d_ty || !d_tz || B < 1) return OPF_EINVAL;
  int rc = net_reserve(n, B);
  if (rc) return rc;
  rc = net_gradients(n, d_x, d_ty, d_tz, B, lambda, loss);
  if (rc) return rc;
  NCU(cudaStreamSynchronize(n->st));
  return OPF_OK;
}

int opf_net_train_step(opf_net_t* n, const float* d_x, const float* d_ty, const float* d_tz, int B,
                       float lambda, float lr, double* loss) {
  int rc = opf_net_gradients(n, d_x, d_ty, d_tz, B, lambda, loss);
  if (rc) return rc;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
  k_adam<<<gs(n->total), 256, 0, n->st>>>(n->P, n->G, n->M1, n->M2, n->total, lr, b1, b2, c1, c2, 1e-8f, n->Pb);
  NCU(cudaStreamSynchronize(n->st));
  NCU(cudaGetLastError());
  return OPF_OK;
}

}  // extern "C"
