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
// with FP32 accumulation on the tcgen05 tensor cores (opf_tcgemm.cu), which
// take row-major K-contiguous operands zero padded to 128-row / 64-column
// multiples; small kernels here lay the operands out that way (im2col rows
// x[b][l + j - 1][c] at column j*C + c, transposes, padded weights).  Master
// weights and Adam moments are FP32.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "opf_internal.h"

namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ operand layouts
// d/dx of gelu(x) = x Phi(x): Phi(x) + x phi(x) (the forward GELU is applied
// in the GEMM epilogue)
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

long pad128(long v) { return (v + 127) / 128 * 128; }
long pad64(long v) { return (v + 63) / 64 * 64; }

// im2col rows: out[m][j*C + c] = x[b][l + s(j-1)][c] (m = b*L + l; s = +1, or
// -1 for the transposed convolution), zero outside 0 <= l' < L, m >= M or
// k >= 3C; out is [Mp][Kp]
__global__ void k_im2col(const bf16* __restrict__ x, int L, int C, int M, int rev, bf16* __restrict__ out, int Mp,
                         int Kp) {
  const long n = (long)Mp * Kp;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int m = (int)(i / Kp), k = (int)(i - (long)m * Kp);
    bf16 v = __float2bfloat16(0.f);
    if (m < M && k < 3 * C) {
      const int j = k / C, c = k - j * C, b = m / L, l = m - b * L;
      const int ls = l + (rev ? 1 - j : j - 1);
      if (ls >= 0 && ls < L) v = x[((long)b * L + ls) * C + c];
    }
    out[i] = v;
  }
}

// The same rows as k_im2col, 8 channels (16 bytes) per thread, one output
// row per grid row (no integer division by the row length): a row of out is
// three shifted rows of x, each C channels, then zeros to Kp.  Needs C and Kp
// multiples of 8 and 16-byte aligned bases (see im2col()).
__global__ void k_im2col8(const bf16* __restrict__ x, int L, int C, int M, int rev, bf16* __restrict__ out, int Kp) {
  const int m = blockIdx.y, k8 = (blockIdx.x * blockDim.x + threadIdx.x) * 8;
  if (k8 >= Kp) return;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (m < M && k8 < 3 * C) {
    const int j = k8 / C, c = k8 - j * C, b = m / L, l = m - b * L;
    const int ls = l + (rev ? 1 - j : j - 1);
    if (ls >= 0 && ls < L) v = *(const uint4*)(x + ((long)b * L + ls) * C + c);
  }
  *(uint4*)(out + (long)m * Kp + k8) = v;
}

int gs(long n);

void im2col(cudaStream_t st, const bf16* x, int L, int C, int M, int rev, bf16* out, int Mp, int Kp) {
  if (C % 8 == 0 && Kp % 8 == 0 && !((uintptr_t)x & 15) && !((uintptr_t)out & 15)) {
    const int kv = Kp / 8;
    k_im2col8<<<dim3((unsigned)((kv + 127) / 128), (unsigned)Mp), 128, 0, st>>>(x, L, C, M, rev, out, Kp);
  } else {
    k_im2col<<<gs((long)Mp * Kp), 256, 0, st>>>(x, L, C, M, rev, out, Mp, Kp);
  }
}

// out[c][r] = src[r][c] (r < R, c < C, row stride lds), zero padded; out is [Cp][Rp]
__global__ void k_transpose(const bf16* __restrict__ src, int R, int C, long lds, bf16* __restrict__ out, int Rp,
                            int Cp) {
  __shared__ bf16 tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + q, c = c0 + threadIdx.x;
    tile[q][threadIdx.x] = (r < R && c < C) ? src[(long)r * lds + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int c = c0 + q, r = r0 + threadIdx.x;
    if (c < Cp && r < Rp) out[(long)c * Rp + r] = tile[threadIdx.x][q];
  }
}

// padded copy: out[r][c] = src[r][c] for r < R, c < C, else 0; out is [Rp][Cp]
__global__ void k_pad(const bf16* __restrict__ src, int R, int C, bf16* __restrict__ out, int Rp, int Cp) {
  const long n = (long)Rp * Cp;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / Cp), c = (int)(i - (long)r * Cp);
    out[i] = (r < R && c < C) ? src[(long)r * C + c] : __float2bfloat16(0.f);
  }
}

// weights of the input-gradient product: out[c][j*Cout + o] = W[o][j*Cin + c]; out is [Cinp][Kp]
__global__ void k_wshift(const bf16* __restrict__ W, int Cout, int Cin, bf16* __restrict__ out, int Cinp, int Kp) {
  const long n = (long)Cinp * Kp;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i / Kp), k = (int)(i - (long)c * Kp);
    bf16 v = __float2bfloat16(0.f);
    if (c < Cin && k < 3 * Cout) {
      const int j = k / Cout, o = k - j * Cout;
      v = W[(long)o * 3 * Cin + (long)j * Cin + c];
    }
    out[i] = v;
  }
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

// column sums (bias gradients): out[n] = sum_m x[m][n]; block (32 columns x
// 32 row groups), partial sums reduced in shared memory
__global__ void __launch_bounds__(1024) k_colsum(const float* __restrict__ x, int M, int N, float* __restrict__ out) {
  __shared__ float part[32][33];
  const int n = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (n < N)
    for (int m = threadIdx.y; m < M; m += 32) s += x[(long)m * N + n];
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && n < N) {
    float t = 0.f;
    for (int q = 0; q < 32; ++q) t += part[q][threadIdx.x];
    out[n] = t;
  }
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
  // GEMM operands (row-major, K contiguous, zero padded): im2col rows of the
  // three layer inputs, their transposes, transposed / shifted output
  // gradients, padded and shifted weights
  bf16 *col[3] = {nullptr, nullptr, nullptr}, *colT = nullptr, *dzT = nullptr, *dzcol = nullptr;
  bf16 *wp[3] = {nullptr, nullptr, nullptr}, *ws[2] = {nullptr, nullptr};
  int* err = nullptr;
  float* gwork = nullptr;  // split-K partial sums of the weight-gradient GEMMs
  long gwork_floats = 0;
  float *pre1 = nullptr, *pre2 = nullptr, *y = nullptr, *dy = nullptr, *dh = nullptr;
  float *pooled = nullptr, *z = nullptr, *dzh = nullptr, *dpooled = nullptr;
  double* sums = nullptr;
  int* aug_idx = nullptr;    // minibatch rows of opf_net_gather_augment (device)
  float* aug_ang = nullptr;  // their shift / rotation phases
  int aug_cap = 0;
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
  for (int i = 0; i < 3; ++i) fr(n->col[i]);
  fr(n->colT), fr(n->dzT), fr(n->dzcol);
  const long BL = (long)B * n->L, W = std::max(n->H, n->Cin);
  const long BLp = pad128(BL), K1 = pad64(3L * n->Cin), K2 = pad64(3L * n->H);
  NCU(cudaMalloc(&n->col[0], BLp * K1 * sizeof(bf16)));
  NCU(cudaMalloc(&n->col[1], BLp * K2 * sizeof(bf16)));
  NCU(cudaMalloc(&n->col[2], BLp * K2 * sizeof(bf16)));
  NCU(cudaMalloc(&n->colT, pad128(3L * W) * BLp * sizeof(bf16)));
  NCU(cudaMalloc(&n->dzT, pad128(W) * BLp * sizeof(bf16)));
  NCU(cudaMalloc(&n->dzcol, BLp * pad64(3L * W) * sizeof(bf16)));
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

// C = A B^T on padded operands with the given epilogue
int gemm(opf_net* n, const bf16* A, const bf16* Bm, int M, int N, int Kp, const opf::TcEpilogue& e) {
  return opf::tc_gemm(A, Bm, M, N, (int)pad128(M), (int)pad128(N), Kp, e, n->err, n->st, n->gwork,
                      n->gwork_floats);
}

opf::TcEpilogue epi(long ldo) {
  opf::TcEpilogue e;
  std::memset(&e, 0, sizeof e);
  e.ldo = ldo;
  return e;
}

// padded copies of the weight matrices (after every parameter change)
void prepare_weights(opf_net* n) {
  const int Ci = n->Cin, H = n->H;
  const int rows[3] = {H, H, Ci}, cols[3] = {3 * Ci, 3 * H, 3 * H};
  for (int i = 0; i < 3; ++i) {
    const long Rp = pad128(rows[i]), Cp = pad64(cols[i]);
    k_pad<<<gs(Rp * Cp), 256, 0, n->st>>>(Pbf(n, 2 * i), rows[i], cols[i], n->wp[i], (int)Rp, (int)Cp);
  }
  // input-gradient weights of layers 3 (Cout = Cin, input H) and 2 (Cout = H, input H)
  k_wshift<<<gs(pad128(H) * pad64(3L * Ci)), 256, 0, n->st>>>(Pbf(n, 4), Ci, H, n->ws[1], (int)pad128(H),
                                                               (int)pad64(3L * Ci));
  k_wshift<<<gs(pad128(H) * pad64(3L * H)), 256, 0, n->st>>>(Pbf(n, 2), H, H, n->ws[0], (int)pad128(H),
                                                              (int)pad64(3L * H));
}

// forward for B samples whose features are at x (f32 [B][L][Cin])
int net_forward(opf_net* n, const float* x, int B) {
  const int L = n->L, Ci = n->Cin, H = n->H, O = n->O;
  const long BL = (long)B * L, BLp = pad128(BL), K1 = pad64(3L * Ci), K2 = pad64(3L * H);
  k_to_bf16<<<gs(BL * Ci), 256, 0, n->st>>>(x, n->xb, BL * Ci);
  int rc;
  // layer 1: h1 = gelu(col(x) W1^T + b1)
  im2col(n->st, n->xb, L, Ci, (int)BL, 0, n->col[0], (int)BLp, (int)K1);
  opf::TcEpilogue e = epi(H);
  e.bias = Pf(n, 1), e.gelu = 1, e.pre_f32 = n->pre1, e.out_bf16 = n->h1;
  if ((rc = gemm(n, n->col[0], n->wp[0], (int)BL, H, (int)K1, e))) return rc;
  // layer 2
  im2col(n->st, n->h1, L, H, (int)BL, 0, n->col[1], (int)BLp, (int)K2);
  e = epi(H);
  e.bias = Pf(n, 3), e.gelu = 1, e.pre_f32 = n->pre2, e.out_bf16 = n->h2;
  if ((rc = gemm(n, n->col[1], n->wp[1], (int)BL, H, (int)K2, e))) return rc;
  // layer 3 (linear)
  im2col(n->st, n->h2, L, H, (int)BL, 0, n->col[2], (int)BLp, (int)K2);
  e = epi(Ci);
  e.bias = Pf(n, 5), e.out_f32 = n->y;
  if ((rc = gemm(n, n->col[2], n->wp[2], (int)BL, Ci, (int)K2, e))) return rc;
  k_pool<<<(B * H + 255) / 256, 256, 0, n->st>>>(n->h2, B, L, H, n->pooled);
  k_head<<<(B * O + 255) / 256, 256, 0, n->st>>>(n->pooled, Pf(n, 6), Pf(n, 7), B, H, O, n->z);
  return OPF_OK;
}

// gradient of one width-3 conv layer (input width Cin, output Cout) given
// dZ (bf16 [BL][Cout], f32 copy dZf) and the layer's im2col rows col:
//   dW[o][k] = sum_m dZ[m][o] col[m][k]        (operands dZ^T, col^T; K = BL)
//   db[o]    = sum_m dZ[m][o]
//   dx[m][c] = sum_{j,o} dZ[(b, l + 1 - j)][o] W[o][j*Cin + c]   (operands col_rev(dZ), ws)
int conv_backward(opf_net* n, int B, const bf16* col, int Kc, int Cin, int Cout, const bf16* dZ, const float* dZf,
                  const bf16* wsh, float* dW, float* db, float* dx) {
  const int L = n->L;
  const long BL = (long)B * L, BLp = pad128(BL);
  int rc;
  dim3 tb(32, 8);
  k_transpose<<<dim3((unsigned)(BLp / 32), (unsigned)(pad128(Cout) / 32)), tb, 0, n->st>>>(
      dZ, (int)BL, Cout, Cout, n->dzT, (int)BLp, (int)pad128(Cout));
  k_transpose<<<dim3((unsigned)(BLp / 32), (unsigned)(pad128(3L * Cin) / 32)), tb, 0, n->st>>>(
      col, (int)BL, 3 * Cin, Kc, n->colT, (int)BLp, (int)pad128(3L * Cin));
  opf::TcEpilogue e = epi(3L * Cin);
  e.out_f32 = dW;
  if ((rc = gemm(n, n->dzT, n->colT, Cout, 3 * Cin, (int)BLp, e))) return rc;
  k_colsum<<<(Cout + 31) / 32, dim3(32, 32), 0, n->st>>>(dZf, (int)BL, Cout, db);
  if (dx) {
    const long Kd = pad64(3L * Cout);
    im2col(n->st, dZ, L, Cout, (int)BL, 1, n->dzcol, (int)BLp, (int)Kd);
    e = epi(Cin);
    e.out_f32 = dx;
    if ((rc = gemm(n, n->dzcol, wsh, (int)BL, Cin, (int)Kd, e))) return rc;
  }
  return OPF_OK;
}

// loss and all parameter gradients into n->G for targets ty [B][L][Cin], tz [B][O]
int net_gradients(opf_net* n, const float* x, const float* ty, const float* tz, int B, float lambda,
                  double* loss) {
  const int L = n->L, Ci = n->Cin, H = n->H, O = n->O;
  const long BL = (long)B * L, K1 = pad64(3L * Ci), K2 = pad64(3L * H);
  int rc = net_forward(n, x, B);
  if (rc) return rc;
  NCU(cudaMemsetAsync(n->sums, 0, 2 * sizeof(double), n->st));
  // dL/dy = 2 (y - ty) / (BL Ci); dL/dz = 2 lambda (z - tz) / (B O)
  k_mse<<<gs(BL * Ci), 256, 0, n->st>>>(n->y, ty, BL * Ci, 1.f / (float)(BL * Ci), n->dy, n->sums);
  k_mse<<<1, 256, 0, n->st>>>(n->z, tz, (long)B * O, lambda / (float)(B * O), n->dzh, n->sums + 1);
  // layer 3 (linear): dZ3 = dy
  k_to_bf16<<<gs(BL * Ci), 256, 0, n->st>>>(n->dy, n->dz, BL * Ci);
  if ((rc = conv_backward(n, B, n->col[2], (int)K2, H, Ci, n->dz, n->dy, n->ws[1], Gf(n, 4), Gf(n, 5), n->dh)))
    return rc;
  // head: pooled mean of h2
  const int hb = (int)std::max<long>((long)O * H, (long)B * H);
  k_head_back<<<(hb + 255) / 256, 256, 0, n->st>>>(n->dzh, n->pooled, Pf(n, 6), B, H, O, Gf(n, 6), Gf(n, 7),
                                                   n->dpooled);
  k_unpool_add<<<gs(BL * H), 256, 0, n->st>>>(n->dpooled, B, L, H, n->dh);
  // layer 2
  k_gelu_back<<<gs(BL * H), 256, 0, n->st>>>(n->dh, n->pre2, n->dz, n->dy, BL * H);
  if ((rc = conv_backward(n, B, n->col[1], (int)K2, H, H, n->dz, n->dy, n->ws[0], Gf(n, 2), Gf(n, 3), n->dh)))
    return rc;
  // layer 1 (input gradient not needed)
  k_gelu_back<<<gs(BL * H), 256, 0, n->st>>>(n->dh, n->pre1, n->dz2, n->dy, BL * H);
  if ((rc = conv_backward(n, B, n->col[0], (int)K1, Ci, H, n->dz2, n->dy, nullptr, Gf(n, 0), Gf(n, 1), nullptr)))
    return rc;
  if (loss) {
    double h[2];
    NCU(cudaMemcpyAsync(h, n->sums, sizeof h, cudaMemcpyDeviceToHost, n->st));
    NCU(cudaStreamSynchronize(n->st));
    *loss = h[0] / (double)(BL * Ci) + lambda * h[1] / (double)(B * O);
  }
  NCU(cudaGetLastError());
  return OPF_OK;
}

// Minibatch gather with the pipe-flow symmetries applied (training-data
// augmentation): sample b is row idx[b] of the device-resident set, its
// complex channel (component, axial index kidx, azimuthal m) turned by
// e^{i (ang[2b] k + ang[2b+1] m)}, k = kidx - (nkf - 1)/2 -- an axial shift
// (ang[2b] = alpha a) and an azimuthal rotation (ang[2b+1] = m_p phi).  The
// head targets are gathered unchanged (period and shift are invariant).
__global__ void k_gather_augment(const float2* __restrict__ x, const float2* __restrict__ y,
                                 const float* __restrict__ z, const int* __restrict__ idx,
                                 const float* __restrict__ ang, int B, int L, int ncomp, int nkf, int mf, int nz,
                                 float2* __restrict__ bx, float2* __restrict__ by, float* __restrict__ bz) {
  const long C = (long)ncomp * nkf * mf;
  const long total = (long)B * L * C;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += stride) {
    const long ch = t % C, bl = t / C;
    const int l = (int)(bl % L), b = (int)(bl / L);
    const int m = (int)(ch % mf), kidx = (int)((ch / mf) % nkf);
    const float ph = ang[2 * b] * (float)(kidx - (nkf - 1) / 2) + ang[2 * b + 1] * (float)m;
    float sn, cs;
    sincosf(ph, &sn, &cs);
    const long src = ((long)idx[b] * L + l) * C + ch, dst = ((long)b * L + l) * C + ch;
    const float2 xv = x[src], yv = y[src];
    bx[dst] = make_float2(xv.x * cs - xv.y * sn, xv.x * sn + xv.y * cs);
    by[dst] = make_float2(yv.x * cs - yv.y * sn, yv.x * sn + yv.y * cs);
  }
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)B * nz; t += stride)
    bz[t] = z[(long)idx[t / nz] * nz + t % nz];
}

void refresh_bf16(opf_net* n) {
  k_to_bf16<<<gs(n->total), 256, 0, n->st>>>(n->P, n->Pb, n->total);
  prepare_weights(n);
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
      cudaMalloc(&n->Pb, t * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc(&n->wp[0], pad128(hidden) * pad64(3L * cin) * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc(&n->wp[1], pad128(hidden) * pad64(3L * hidden) * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc(&n->wp[2], pad128(cin) * pad64(3L * hidden) * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc(&n->ws[0], pad128(hidden) * pad64(3L * hidden) * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc(&n->ws[1], pad128(hidden) * pad64(3L * cin) * sizeof(bf16)) != cudaSuccess ||
      cudaMalloc(&n->err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&n->gwork, (n->gwork_floats = 8L * std::max(3L * hidden * std::max(cin, hidden), 1L)) *
                                sizeof(float)) != cudaSuccess) {
    opf::set_last_error("opf_net_create: device allocation failed");
    opf_net_destroy(n);
    return nullptr;
  }
  cudaMemcpy(n->P, h.data(), t * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(n->G, 0, t * sizeof(float));
  cudaMemset(n->M1, 0, t * sizeof(float));
  cudaMemset(n->M2, 0, t * sizeof(float));
  cudaMemset(n->err, 0, sizeof(int));
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
                  (void*)n->dpooled, (void*)n->sums, (void*)n->col[0], (void*)n->col[1], (void*)n->col[2],
                  (void*)n->colT, (void*)n->dzT, (void*)n->dzcol, (void*)n->wp[0], (void*)n->wp[1],
                  (void*)n->wp[2], (void*)n->ws[0], (void*)n->ws[1], (void*)n->err, (void*)n->gwork,
                  (void*)n->aug_idx, (void*)n->aug_ang})
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

// a tensor-core GEMM whose bounded wait ran out leaves the flag set
static int net_check(opf_net_t* n) {
  int h = 0;
  NCU(cudaMemcpy(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(n->err, 0, sizeof(int));
    opf::set_last_error("proposal network: a tensor-core GEMM timed out waiting for its operands");
    return OPF_ETIMEOUT;
  }
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
  return net_check(n);
}

int opf_net_gradients(opf_net_t* n, const float* d_x, const float* d_ty, const float* d_tz, int B,
                      float lambda, double* loss) {
  if (!n || !d_x || !d_ty || !d_tz || B < 1) return OPF_EINVAL;
  int rc = net_reserve(n, B);
  if (rc) return rc;
  rc = net_gradients(n, d_x, d_ty, d_tz, B, lambda, loss);
  if (rc) return rc;
  NCU(cudaStreamSynchronize(n->st));
  return net_check(n);
}

int opf_net_train_step(opf_net_t* n, const float* d_x, const float* d_ty, const float* d_tz, int B,
                       float lambda, float lr, double* loss) {
  int rc = opf_net_gradients(n, d_x, d_ty, d_tz, B, lambda, loss);
  if (rc) return rc;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
  k_adam<<<gs(n->total), 256, 0, n->st>>>(n->P, n->G, n->M1, n->M2, n->total, lr, b1, b2, c1, c2, 1e-8f, n->Pb);
  prepare_weights(n);
  NCU(cudaStreamSynchronize(n->st));
  NCU(cudaGetLastError());
  return OPF_OK;
}

int opf_net_gather_augment(opf_net_t* n, int B, int L, int ncomp, int nkf, int mf, int nz, const float* d_x,
                           const float* d_y, const float* d_z, long rows, const int* idx, const float* ang,
                           float* d_bx, float* d_by, float* d_bz) {
  if (!n || B < 1 || L < 1 || ncomp < 1 || nkf < 1 || mf < 1 || nz < 1 || rows < 1 || !d_x || !d_y || !d_z ||
      !idx || !ang || !d_bx || !d_by || !d_bz) {
    opf::set_last_error("opf_net_gather_augment: bad arguments");
    return OPF_EINVAL;
  }
  for (int b = 0; b < B; ++b)
    if (idx[b] < 0 || idx[b] >= rows) {
      opf::set_last_error("opf_net_gather_augment: sample index out of range");
      return OPF_EINVAL;
    }
  if (n->aug_cap < B) {
    if (n->aug_idx) cudaFree(n->aug_idx);
    if (n->aug_ang) cudaFree(n->aug_ang);
    n->aug_idx = nullptr;
    n->aug_ang = nullptr;
    n->aug_cap = 0;
    NCU(cudaMalloc((void**)&n->aug_idx, (size_t)B * sizeof(int)));
    NCU(cudaMalloc((void**)&n->aug_ang, (size_t)2 * B * sizeof(float)));
    n->aug_cap = B;
  }
  NCU(cudaMemcpyAsync(n->aug_idx, idx, (size_t)B * sizeof(int), cudaMemcpyHostToDevice, n->st));
  NCU(cudaMemcpyAsync(n->aug_ang, ang, (size_t)2 * B * sizeof(float), cudaMemcpyHostToDevice, n->st));
  const long total = (long)B * L * ncomp * nkf * mf;
  k_gather_augment<<<gs(total), 256, 0, n->st>>>((const float2*)d_x, (const float2*)d_y, d_z, n->aug_idx,
                                                 n->aug_ang, B, L, ncomp, nkf, mf, nz, (float2*)d_bx,
                                                 (float2*)d_by, d_bz);
  NCU(cudaGetLastError());
  return OPF_OK;
}

}  // extern "C"
