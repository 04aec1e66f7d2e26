// Device kernels of the pipe-flow time step (paper section 2).
//
// Nonlinear term (section 2.2, evaluated pseudo-spectrally):
//   k_curl      spectral u+-, u_z -> (u_r, u_theta, u_z, w_r, w_theta, w_z)
//   k_zsynth    inverse FFT in z (2K-1 modes zero-padded to 3K points)
//   k_product   per (r, z) row: C2R in theta (M modes -> 3M points), u x w,
//               R2C in theta keeping m < M
//   k_zanalysis forward FFT in z keeping |k| < K, 1/(3K 3M) scaling,
//               (N_r, N_theta) -> N+-, base forcing 4/Re on the (0,0) mode
// Linear part (section 2.2, banded LU per Fourier mode; section 2 influence
// matrix): k_solve, one block per tile of T modes at fixed m.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>

#include "opf_fft.cuh"
#include "opf_internal.h"

namespace opf {

__device__ __forceinline__ int row_lo_d(int i, int N) { return min(max(i - 4, 0), N - 9); }

// Programmatic dependent launch between the kernels of a step: each step
// kernel lets its successor launch once all of its own blocks have reached
// the trigger (d.pdl = 1: at the top; 2: before the final store phase), and
// waits for its predecessor grid to complete -- with its memory visible --
// before it reads or writes any buffer another kernel of the step touches
// (grid_dep_wait after a prologue that reads only setup data: twiddles,
// stencils, factors).  Every step kernel waits, so the ordering is
// transitive along the stream.  Without a programmatic launch both are
// no-ops.
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger_at(const Dims& d, int where) {
  if (d.pdl == where) grid_dep_trigger();
}
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with the programmatic-serialisation attribute when d.pdl is set
// (captured into a graph, the edge to the previous kernel becomes a
// programmatic dependency), plainly otherwise.
template <typename... KArgs, typename... Args>
void launch_step_kernel(const Dims& d, void (*kern)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t st,
                        Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = d.pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Batched launches: trajectory b = blockIdx.z; its buffers sit `stride` bytes
// after trajectory b-1's (stride 0: shared).  Null stays null.
template <typename P>
__device__ __forceinline__ P* bofs(P* p, long stride) {
  return p ? (P*)((char*)p + (long)blockIdx.z * stride) : p;
}

// ------------------------------------------------------------------ ABI <-> internal
// abi: [3][M][nk][N] (u_r, u_theta, u_z); internal: [3][M][N][nk] (u+, u-, u_z).
// flag (optional): a non-zero value there (set by the NaN check launched
// before) leaves U as it is; beta (optional) is reset to 0 otherwise.
// nan_out (optional): set to 1 if any coefficient read is not finite (every
// coefficient is read by the thread of its own (m, k, n)).
// herm (optional, zeroed by the caller): herm[0], herm[1] become the upper 32
// bits of max |A(k,0) - conj A(-k,0)| and of max |A(k,0)| over the m = 0
// coefficients (real and imaginary parts separately, all three components):
// the upper word of a non-negative double orders like the double, and keeps
// it to 2^-20 relative.
__global__ void k_abi_to_internal(Dims d, const double2* __restrict__ abi, double2* __restrict__ U,
                                  const int* __restrict__ flag, double* __restrict__ beta, int* nan_out,
                                  unsigned* herm) {
  if (flag && *flag) return;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (beta && idx == 0) *beta = 0.0;
  if (idx >= d.F) return;
  const int n = idx % d.N;
  const long t = idx / d.N;
  const int kk = t % d.nk;
  const int m = t / d.nk;
  const long fs = d.F;
  auto ld = [&](int c, int kq) { return abi[c * fs + ((long)m * d.nk + kq) * d.N + n]; };
  double2 ur = ld(0, kk), ut = ld(1, kk), uz = ld(2, kk);
  if (nan_out && !(isfinite(ur.x) && isfinite(ur.y) && isfinite(ut.x) && isfinite(ut.y) && isfinite(uz.x) &&
                   isfinite(uz.y)))
    atomicOr(nan_out, 1);
  if (m == 0) {  // Hermitian projection A(-k,0) = conj A(k,0)
    const int kq = d.nk - 1 - kk;
    const double2 vr = ld(0, kq), vt = ld(1, kq), vz = ld(2, kq);
    if (herm) {
      const double asym = fmax(fmax(fmax(fabs(ur.x - vr.x), fabs(ur.y + vr.y)),
                                    fmax(fabs(ut.x - vt.x), fabs(ut.y + vt.y))),
                               fmax(fabs(uz.x - vz.x), fabs(uz.y + vz.y)));
      const double amp = fmax(fmax(fmax(fabs(ur.x), fabs(ur.y)), fmax(fabs(ut.x), fabs(ut.y))),
                              fmax(fabs(uz.x), fabs(uz.y)));
      const unsigned lanes = __activemask();
      const unsigned ha = __reduce_max_sync(lanes, (unsigned)(__double_as_longlong(asym) >> 32));
      const unsigned hm = __reduce_max_sync(lanes, (unsigned)(__double_as_longlong(amp) >> 32));
      if ((int)(threadIdx.x & 31) == __ffs(lanes) - 1) {
        atomicMax(herm, ha);
        atomicMax(herm + 1, hm);
      }
    }
    ur = double2{0.5 * (ur.x + vr.x), 0.5 * (ur.y - vr.y)};
    ut = double2{0.5 * (ut.x + vt.x), 0.5 * (ut.y - vt.y)};
    uz = double2{0.5 * (uz.x + vz.x), 0.5 * (uz.y - vz.y)};
  }
  const long o = ((long)m * d.N + n) * d.nk + kk;
  U[0 * fs + o] = double2{ur.x - ut.y, ur.y + ut.x};  // u+ = u_r + i u_theta
  U[1 * fs + o] = double2{ur.x + ut.y, ur.y - ut.x};  // u- = u_r - i u_theta
  U[2 * fs + o] = uz;
}

__global__ void k_internal_to_abi(Dims d, const double2* __restrict__ U, double2* __restrict__ abi) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.F) return;
  const int n = idx % d.N;
  const long t = idx / d.N;
  const int kk = t % d.nk;
  const int m = t / d.nk;
  const long fs = d.F;
  const long i = ((long)m * d.N + n) * d.nk + kk;
  const double2 a = U[i], b = U[fs + i];
  const long o = ((long)m * d.nk + kk) * d.N + n;
  abi[o] = double2{0.5 * (a.x + b.x), 0.5 * (a.y + b.y)};           // u_r
  abi[fs + o] = double2{0.5 * (a.y - b.y), -0.5 * (a.x - b.x)};      // u_theta
  abi[2 * fs + o] = U[2 * fs + i];
}

void launch_abi_to_internal(const Dims& d, const double2* abi, double2* U, cudaStream_t st, const int* flag,
                            double* beta, int* nan_out, unsigned* herm) {
  const int nb = (int)((d.F + 255) / 256);
  k_abi_to_internal<<<nb, 256, 0, st>>>(d, abi, U, flag, beta, nan_out, herm);
}

// dst = src (n double2) unless *flag is set; beta reset to 0 with it
__global__ void k_copy_unless(const double2* __restrict__ src, double2* __restrict__ dst, long n,
                              const int* __restrict__ flag, double* __restrict__ beta) {
  if (*flag) return;
  const long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (beta && i0 == 0) *beta = 0.0;
  for (long i = i0; i < n; i += (long)gridDim.x * blockDim.x) dst[i] = src[i];
}

void launch_copy_unless(const double2* src, double2* dst, long n, const int* flag, double* beta,
                        cudaStream_t st) {
  const int nb = (int)std::min<long>((n + 255) / 256, 4L * 152);
  k_copy_unless<<<nb, 256, 0, st>>>(src, dst, n, flag, beta);
}
void launch_internal_to_abi(const Dims& d, const double2* U, double2* abi, int, cudaStream_t st) {
  const int nb = (int)((d.F + 255) / 256);
  k_internal_to_abi<<<nb, 256, 0, st>>>(d, U, abi);
}

// ------------------------------------------------------------------ curl (A1)
// The radial columns of a trajectory -- column (m, kk), all N rows -- are
// split into contiguous runs of whole columns, one per block (their count
// differing by at most one between blocks).  A block stages its columns --
// each u+-, u_z value read once, u_r and u_theta formed in FP64 -- in shared
// memory, and the 9-point radial stencils read their neighbours from there.
// Threads take the block's points row by row with the columns innermost, so
// that a warp's stencil rows are shared by the lanes of one row and its
// stores run along k.  Columns per block: on a grid of a few waves, the
// count that puts the fewest warp-passes on the busiest SM (then the most
// resident warps; the grid of four columns per block of a one-wave medium
// trajectory left a third of the SMs' time idle), else four.
//
// SPLIT (mixed precision): the laminar base flow U = (1 - r^2) z,
// Omega = 2r theta is removed in FP64 (W6 then holds u', w' in FP32), and the
// terms linear in the perturbation, U x w' + u' x Omega (+ U x Omega on
// (0,0)), are evaluated here per mode in FP64 -- they are diagonal in r -- and
// written to Nlin in +- form.  FP64 arithmetic is kept to what Nlin needs (the
// u_z derivative, w_r, w_theta); the u_theta derivative feeds only w_z, which
// goes to the FP32 product, and is taken in FP32 from an FP32 copy of the
// u_theta tile.  The factor 1/2 of u_r = (u+ + u-)/2 and
// u_theta = (u+ - u-)/(2i) goes into the constants that multiply them (exact
// scalings by two, so the results are those of the halved values).  Without
// SPLIT everything is FP64.
constexpr int kCurlThreads = 128;

static int device_sms() {
  static const int sms = [] {
    int dev = 0, n = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
  }();
  return sms;
}

// Blocks per trajectory and the most columns one block takes.
struct CurlShape {
  int nbx, kc;
};
static CurlShape curl_shape(const Dims& d) {
  const long sms = device_sms();
  const long cols = (long)d.M * d.nk, B = d.B > 0 ? d.B : 1, N = d.N;
  const long warps_max = kCurlThreads / 32;
  long cpb = 4;
  if ((cols + 3) / 4 * B <= 8 * sms) {
    long best_cost = -1, best_conc = 0;
    for (long c = 1; c <= 16 && c <= cols; ++c) {
      const long w = (c * N + 31) / 32;  // warp-passes of a block
      if (c * N < 32 || w > 4 * warps_max) continue;
      const long per_sm = ((cols + c - 1) / c * B + sms - 1) / sms;
      const long cost = per_sm * w, conc = per_sm * std::min(w, warps_max);
      if (best_cost < 0 || cost < best_cost || (cost == best_cost && conc > best_conc)) {
        best_cost = cost;
        best_conc = conc;
        cpb = c;
      }
    }
  }
  cpb = std::min(cpb, cols);
  const long nbx = (cols + cpb - 1) / cpb;
  return CurlShape{(int)nbx, (int)((cols + nbx - 1) / nbx)};
}

size_t curl_smem(const Dims& d) {
  const size_t kc = (size_t)curl_shape(d).kc, N = (size_t)d.N;
  return N * kc * (3 * sizeof(double2) + sizeof(float2)) + kc * sizeof(double) + 2 * N * sizeof(double) +
         2 * kc * sizeof(int);
}

// One grid point (m, kk, radial row n) of A1 from the radial column of its
// mode: uz_at(i), ut_at(i) (FP64) and ut32_at(i) (FP32, SPLIT) give u_z and
// u_theta at row i; ur, ut, uz are the point's own values; ak = alpha k.
// SPLIT with SUMS: ur and ut are 2 u_r and 2 u_theta, ak is alpha k / 2, and
// Ub, Ob are U = 1 - r^2 and Omega = 2r at the point's row (else formed
// here from r).  d1 = [2][N][9] stencils, d1f =
// the FP32 stencils then FP32 1/r, rr and rinv the radial points and their
// inverses (all of this trajectory).  Writes the six W6 components (and,
// SPLIT, the FP64 linear terms Nlin in +- form).
template <typename V, bool SPLIT, bool SUMS = false, typename UzAt, typename UtAt, typename Ut32At>
__device__ __forceinline__ void curl_point(const Dims& d, int m, int kk, int n, double ak,
                                           const double* __restrict__ d1, const float* __restrict__ d1f,
                                           const double* __restrict__ rr, const double* __restrict__ rinv,
                                           UzAt uz_at, UtAt ut_at, Ut32At ut32_at, double2 ur, double2 ut,
                                           double2 uz, V* __restrict__ W6, double2* __restrict__ Nlin,
                                           double Ub = 0.0, double Ob = 0.0) {
  using T = typename Scalar<V>::T;
  const int N = d.N, nk = d.nk;
  const long fs = d.F;
  const int mt = d.m_p * m;
  const int ps = mt & 1, pv = ps ^ 1;
  const int lo = row_lo_d(n, N);
  const double* ws = d1 + ((long)ps * N + n) * 9;
  double dzx = 0, dzy = 0;  // d/dr of u_z (FP64)
  T dtx = 0, dty = 0;       // d/dr of u_theta
  if constexpr (SPLIT) {
    const float* wv = d1f + ((long)pv * N + n) * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const double2 z = uz_at(lo + q);
      const float2 t = ut32_at(lo + q);
      dzx = fma(ws[q], z.x, dzx);
      dzy = fma(ws[q], z.y, dzy);
      dtx = fmaf(wv[q], t.x, dtx);
      dty = fmaf(wv[q], t.y, dty);
    }
  } else {
    const double* wv = d1 + ((long)pv * N + n) * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const double2 z = uz_at(lo + q), t = ut_at(lo + q);
      dzx = fma(ws[q], z.x, dzx);
      dzy = fma(ws[q], z.y, dzy);
      dtx = fma(wv[q], t.x, dtx);
      dty = fma(wv[q], t.y, dty);
    }
  }
  const double ri = rinv[n];
  const double mri = mt * ri;
  // w_r = i (m~ u_z / r - ak u_theta)
  const double xr = mri * uz.x - ak * ut.x, xi = mri * uz.y - ak * ut.y;
  // w_theta = i ak u_r - d_r u_z
  double wtx = -ak * ur.y - dzx, wty = ak * ur.x - dzy;
  const long w = ((long)m * N + n) * nk + kk;
  double uzx = uz.x;
  if constexpr (SPLIT) {
    if constexpr (!SUMS) {
      const double r = rr[n];
      Ub = 1.0 - r * r;
      Ob = 2.0 * r;
    }
    const bool mean = (m == 0 && kk == d.K - 1);
    if (mean) {
      uzx -= Ub;
      wtx -= Ob;
    }
    // N_r = -U w'_t - Omega u'_z, N_t = U w'_r, N_z = Omega u'_r
    double nrx = -Ub * wtx - Ob * uzx, nry = -Ub * wty - Ob * uz.y;
    if (mean) nrx -= Ub * Ob;
    const double ntx = Ub * (-xi), nty = Ub * xr;
    Nlin[w] = double2{nrx - nty, nry + ntx};
    double2 nminus = double2{nrx + nty, nry - ntx};
    if (d.rotate && mt == 1 && kk == d.K - 1) {  // Coriolis force of U z: N- = -2 U (Omega_y + i Omega_x)
      nminus.x -= 2.0 * Ub * d.rot_y;
      nminus.y -= 2.0 * Ub * d.rot_x;
    }
    Nlin[fs + w] = nminus;
    if constexpr (SUMS) {
      const double r = rr[n];  // Omega u_r = r (2 u_r)
      Nlin[2 * fs + w] = double2{r * ur.x, r * ur.y};
    } else {
      Nlin[2 * fs + w] = double2{Ob * ur.x, Ob * ur.y};
    }
    // w_z = d_r u_theta + u_theta / r - i m~ u_r / r, in FP32
    const float ri32 = d1f[2 * 9 * N + n], mri32 = (float)mt * ri32;
    const float2 ut32 = ut32_at(n);
    const float urx = SUMS ? 0.5f * (float)ur.x : (float)ur.x, ury = SUMS ? 0.5f * (float)ur.y : (float)ur.y;
    W6[0 * fs + w] = float2{urx, ury};
    W6[1 * fs + w] = ut32;
    W6[2 * fs + w] = float2{(float)uzx, (float)uz.y};
    W6[3 * fs + w] = float2{(float)(-xi), (float)xr};
    W6[4 * fs + w] = float2{(float)wtx, (float)wty};
    W6[5 * fs + w] = float2{fmaf(mri32, ury, fmaf(ri32, ut32.x, dtx)), fmaf(-mri32, urx, fmaf(ri32, ut32.y, dty))};
  } else {
    W6[0 * fs + w] = ur;
    W6[1 * fs + w] = ut;
    W6[2 * fs + w] = uz;
    W6[3 * fs + w] = V{-xi, xr};
    W6[4 * fs + w] = V{wtx, wty};
    W6[5 * fs + w] = V{dtx + ri * ut.x + mri * ur.y, dty + ri * ut.y - mri * ur.x};
  }
}

// kc: the most columns of a block (curl_shape), the shared-memory size.
template <typename V, bool SPLIT>
__global__ void __launch_bounds__(kCurlThreads) k_curl(Dims d, int kc, const double* __restrict__ d1,
                                                       const float* __restrict__ d1f, const double* __restrict__ rr,
                                                       const double* __restrict__ rinv,
                                                       const double2* __restrict__ U, V* __restrict__ W6,
                                                       double2* __restrict__ Nlin) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = d.N, nk = d.nk;
  double2* s_uz = (double2*)smraw;            // [N][ncb] u_z
  double2* s_ur = s_uz + N * kc;              // [N][ncb] u_r (SPLIT: 2 u_r)
  double2* s_ut = s_ur + N * kc;              // [N][ncb] u_theta (SPLIT: 2 u_theta)
  float2* s_ut32 = (float2*)(s_ut + N * kc);  // [N][ncb] u_theta in FP32 (SPLIT)
  double* s_ak = (double*)(s_ut32 + N * kc);  // [ncb] alpha k of the columns (SPLIT: alpha k / 2)
  double* s_ub = s_ak + kc;                   // [N] U = 1 - r^2 (SPLIT)
  double* s_ob = s_ub + N;                    // [N] Omega = 2r (SPLIT)
  int* s_m = (int*)(s_ob + N);                // [ncb] m of the columns
  int* s_kk = s_m + kc;                       // [ncb] kk of the columns
  d1 = bofs(d1, d.ps);
  d1f = bofs(d1f, d.ps);
  rr = bofs(rr, d.ps);
  rinv = bofs(rinv, d.ps);
  U = bofs(U, d.ss);
  W6 = bofs(W6, d.ss);
  Nlin = bofs(Nlin, d.ss);
  const long fs = d.F, cols = (long)d.M * nk;
  const int col0 = (int)((long)blockIdx.x * cols / gridDim.x);
  const int ncb = (int)((long)(blockIdx.x + 1) * cols / gridDim.x) - col0;  // this block's columns, <= kc
  grid_dep_trigger_at(d, 1);
  if (ncb <= 0) return;
  for (int c = threadIdx.x; c < ncb; c += blockDim.x) {
    const int col = col0 + c, m = col / nk, kk = col - m * nk;
    s_m[c] = m;
    s_kk[c] = kk;
    const double ak = d.alpha * (kk - (d.K - 1));
    s_ak[c] = SPLIT ? 0.5 * ak : ak;
  }
  if constexpr (SPLIT)
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      const double r = rr[n];
      s_ub[n] = 1.0 - r * r;
      s_ob[n] = 2.0 * r;
    }
  __syncthreads();
  grid_dep_wait();
  for (int e = threadIdx.x; e < N * ncb; e += blockDim.x) {
    const int n = e / ncb, c = e - n * ncb;
    const long o = ((long)s_m[c] * N + n) * nk + s_kk[c];
    const double2 a = U[o], b = U[fs + o];
    s_uz[e] = U[2 * fs + o];
    if constexpr (SPLIT) {
      const double2 ut2 = double2{a.y - b.y, b.x - a.x};
      s_ur[e] = double2{a.x + b.x, a.y + b.y};
      s_ut[e] = ut2;
      s_ut32[e] = float2{0.5f * (float)ut2.x, 0.5f * (float)ut2.y};
    } else {
      s_ur[e] = double2{0.5 * (a.x + b.x), 0.5 * (a.y + b.y)};
      s_ut[e] = double2{0.5 * (a.y - b.y), -0.5 * (a.x - b.x)};
    }
  }
  __syncthreads();
  grid_dep_trigger_at(d, 2);
  for (int e = threadIdx.x; e < N * ncb; e += blockDim.x) {
    const int n = e / ncb, c = e - n * ncb;
    const double2 *cz = s_uz + c, *ct = s_ut + c;
    const float2* ct32 = s_ut32 + c;
    curl_point<V, SPLIT, true>(
        d, s_m[c], s_kk[c], n, s_ak[c], d1, d1f, rr, rinv, [=](int i) { return cz[i * ncb]; },
        [=](int i) { return ct[i * ncb]; }, [=](int i) { return ct32[i * ncb]; }, s_ur[e], s_ut[e], s_uz[e], W6,
        Nlin, SPLIT ? s_ub[n] : 0.0, SPLIT ? s_ob[n] : 0.0);
  }
}

void launch_curl(const Dims& d, const DevSetup& s, const double2* U, double2* W6, cudaStream_t st) {
  const CurlShape c = curl_shape(d);
  launch_step_kernel(d, k_curl<double2, false>, dim3(c.nbx, 1, d.B), dim3(kCurlThreads), curl_smem(d), st, d,
                     c.kc, (const double*)s.d1, (const float*)nullptr, (const double*)nullptr,
                     (const double*)s.rinv, U, W6, (double2*)nullptr);
}

void launch_curl_split32(const Dims& d, const DevSetup& s, const double2* U, float2* W6,
                         double2* Nlin, cudaStream_t st) {
  const CurlShape c = curl_shape(d);
  launch_step_kernel(d, k_curl<float2, true>, dim3(c.nbx, 1, d.B), dim3(kCurlThreads), curl_smem(d), st, d,
                     c.kc, (const double*)s.d1, (const float*)s.d1f, (const double*)s.r,
                     (const double*)s.rinv, U, W6, Nlin);
}

// Threads per block of the transform kernels: 256 for grids of at most four
// blocks per SM (a single wave of few blocks: more threads per batch of
// sequences shorten each block's passes), 128 for larger grids, which
// measured as fast or faster in the smaller unit.  The arithmetic is the
// same either way.
static unsigned transform_threads(const dim3& g) {
  return (long)g.x * g.y * g.z <= 4L * device_sms() ? 256u : 128u;
}

// ------------------------------------------------------------------ z synthesis (A2)

// NZ > 0: the z length 3K is the compile-time constant NZ (compiled plan).
template <typename V, int NZ>
__global__ void __launch_bounds__(256) k_zsynth(Dims d, FftPlan pz, const V* __restrict__ twz,
                                                const V* __restrict__ W6, V* __restrict__ Z6) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nz = NZ > 0 ? NZ : d.nz, ld = nz + 1, MC = d.mcz;
  V* A = (V*)smraw;
  V* B = A + MC * ld;
  V* tw = B + MC * ld;
  const int m0 = blockIdx.x * MC, n = blockIdx.y / 6, f = blockIdx.y % 6;
  const int K = d.K;
  twz = bofs(twz, d.ps);
  W6 = bofs(W6, d.ss);
  Z6 = bofs(Z6, d.ss);
  grid_dep_trigger_at(d, 1);
  for (int e = threadIdx.x; e < nz; e += blockDim.x) tw[e] = twz[e];
  const long fs = d.F;
  grid_dep_wait();
  block_copy_batched<8, V>(
      MC * nz,
      [&](int e) {
        const int z = e % nz, m = m0 + e / nz;
        const int k = z < K ? z : z - nz;
        V v = V{0, 0};
        if (m < d.M && (z < K || z > nz - K)) v = W6[f * fs + ((long)m * d.N + n) * d.nk + k + K - 1];
        return v;
      },
      [&](int e, V v) { A[(e / nz) * ld + e % nz] = v; });
  __syncthreads();
  const V* res;
  if constexpr (NZ > 0) res = block_fft_c<NZ, +1, true>(A, B, MC, ld, tw);
  else res = block_fft(A, B, MC, ld, pz, tw, +1);
  const int mcn = min(MC, d.M - m0);
  grid_dep_trigger_at(d, 2);
  for (int e = threadIdx.x; e < mcn * nz; e += blockDim.x) {
    const int mc = e % mcn, z = e / mcn;
    Z6[(((long)f * d.N + n) * nz + z) * d.M + m0 + mc] = res[mc * ld + z];
  }
}

size_t zsynth_smem(const Dims& d, int mc, size_t vb) { return (2 * (size_t)mc * (d.nz + 1) + d.nz) * vb; }

void launch_zsynth32(const Dims& d, const DevSetup& s, const FftPlan& pz, const float2* W6,
                     float2* Z6, cudaStream_t st) {
  dim3 g((d.M + d.mcz - 1) / d.mcz, d.N * 6, d.B);
  const size_t sm = zsynth_smem(d, d.mcz, sizeof(float2));
  with_fft_length(d.nz, [&](auto n) {
    launch_step_kernel(d, k_zsynth<float2, decltype(n)::value>, g, dim3(transform_threads(g)), sm, st, d, pz,
                       (const float2*)s.tw_z32, W6, Z6);
  });
}

void launch_zsynth(const Dims& d, const DevSetup& s, const FftPlan& pz, const double2* W6,
                   double2* Z6, cudaStream_t st) {
  dim3 g((d.M + d.mcz - 1) / d.mcz, d.N * 6, d.B);
  const size_t sm = zsynth_smem(d, d.mcz, sizeof(double2));
  with_fft_length(d.nz, [&](auto n) {
    launch_step_kernel(d, k_zsynth<double2, decltype(n)::value>, g, dim3(transform_threads(g)), sm, st, d, pz,
                       (const double2*)s.tw_z, W6, Z6);
  });
}

// ------------------------------------------------------------------ product (A3)

__device__ __forceinline__ void sincos_pi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincos_pi(float x, float* s, float* c) { sincospif(x, s, c); }

// NTH > 0: the theta length 3M is the compile-time constant NTH.
template <typename V, int NTH>
__global__ void __launch_bounds__(256) k_product(Dims d, FftPlan pth, const V* __restrict__ twth,
                                                 const V* __restrict__ Z6, V* __restrict__ ZN) {
  using T = typename Scalar<V>::T;
  // FP64: the real N_z of two z rows go through one complex forward
  // transform (1.5 instead of 2 transforms per row on the FP64 pipe); the
  // FP32 path keeps one per row, the arithmetic of the fused launch
  constexpr bool kPackNz = sizeof(T) == 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nth = NTH > 0 ? NTH : d.nth, ld = nth, M = d.M;
  const int ZC = d.zc;
  V* A = (V*)smraw;            // 3 * ZC sequences
  V* B = A + 3 * ZC * ld;      // 3 * ZC sequences
  V* tw = B + 3 * ZC * ld;
  const int z0 = blockIdx.x * ZC, n = blockIdx.y, nz = d.nz;
  const int zc = min(ZC, nz - z0);
  twth = bofs(twth, d.ps);
  Z6 = bofs(Z6, d.ss);
  ZN = bofs(ZN, d.ss);
  grid_dep_trigger_at(d, 1);
  for (int e = threadIdx.x; e < nth; e += blockDim.x) tw[e] = twth[e];
  const long fstride = (long)d.N * nz * M;
  grid_dep_wait();
  // spectra of the pairs (u_r,u_t), (u_z,w_r), (w_t,w_z):  Z = A + i B
  block_copy_batched<8, V>(
      zc * 3 * nth,
      [&](int e) {
        const int q = e % nth, pr = (e / nth) % 3, zr = e / (3 * nth);
        const long rowa = ((long)(2 * pr) * d.N + n) * nz + z0 + zr;
        V v = V{0, 0};
        if (q < M) {
          V a = Z6[rowa * M + q], b = Z6[(rowa + (long)d.N * nz) * M + q];
          if (q == 0) { a.y = 0; b.y = 0; }
          v = V{a.x - b.y, a.y + b.x};
        } else if (q > nth - M) {
          const int m = nth - q;
          const V a = Z6[rowa * M + m], b = Z6[(rowa + (long)d.N * nz) * M + m];
          v = V{a.x + b.y, -a.y + b.x};  // conj(a) + i conj(b)
        }
        return v;
      },
      [&](int e, V v) { A[(e / nth) * ld + e % nth] = v; });
  __syncthreads();
  V* res;
  if constexpr (NTH > 0) res = block_fft_c<NTH, +1, true>(A, B, 3 * zc, ld, tw);
  else res = block_fft(A, B, 3 * zc, ld, pth, tw, +1);
  V* C = (res == A) ? B : A;
  // CFL number of this radial plane (optional): max over the grid of
  // |u_r|/dr, |u_t|/(r dtheta), |u_z|/dz for the TOTAL velocity (the FP32
  // path carries the perturbation only, so the laminar 1 - r^2 is added back)
  // (taken in the transform precision T)
  double* cfl = bofs(d.cfl, d.ss);
  T inv_dr = 0, inv_rdt = 0, inv_dz = 0, Ubase = 0;
  if (cfl) {
    const double* rinv = bofs(d.rinv_cfl, d.ps);
    const T one = 1, rn = one / (T)rinv[n];
    const T rm = n > 0 ? one / (T)rinv[n - 1] : -rn;
    const T rp = n < d.N - 1 ? one / (T)rinv[n + 1] : one + (one - rm);
    const T twopi = (T)6.283185307179586;
    inv_dr = one / fmin(rn - rm, rp - rn);
    inv_rdt = (T)(d.m_p * nth) / (twopi * rn);
    inv_dz = (T)d.alpha * (T)nz / twopi;
    if constexpr (sizeof(T) == 4) Ubase = one - rn * rn;
  }
  T cmax = 0;
  for (int e = threadIdx.x; e < zc * nth; e += blockDim.x) {
    const int q = e % nth, zr = e / nth;
    const V x0 = res[(zr * 3 + 0) * ld + q], x1 = res[(zr * 3 + 1) * ld + q], x2 = res[(zr * 3 + 2) * ld + q];
    const T ur = x0.x, ut = x0.y, uz = x1.x, wr = x1.y, wt = x2.x, wz = x2.y;
    T nr = ut * wz - uz * wt, nt = uz * wr - ur * wz, nz = ur * wt - ut * wr;
    if (d.rotate) {  // Coriolis -2 Omega x u, Omega in cylindrical components at theta_q
      T sn, cs;
      sincos_pi((T)(2 * q) / (T)(d.m_p * nth), &sn, &cs);
      const T rx = (T)d.rot_x, ry = (T)d.rot_y;
      const T o_r = rx * cs + ry * sn, o_t = -rx * sn + ry * cs;
      const T o_z = (T)d.rot_z;
      nr -= (T)2 * (o_t * uz - o_z * ut);
      nt -= (T)2 * (o_z * ur - o_r * uz);
      nz -= (T)2 * (o_r * ut - o_t * ur);
    }
    if constexpr (kPackNz) {  // rows zr, zr^1 share one sequence for N_z: re <- even row, im <- odd row
      C[zr * ld + q] = V{nr, nt};
      T* pz = (T*)&C[(zc + (zr >> 1)) * ld + q];
      pz[zr & 1] = nz;
      if ((zc & 1) && zr == zc - 1) pz[1] = (T)0;  // the last row of an odd count has no partner
    } else {
      C[(zr * 2 + 0) * ld + q] = V{nr, nt};
      C[(zr * 2 + 1) * ld + q] = V{nz, (T)0};
    }
    if (cfl) cmax = fmax(cmax, fmax(fabs(ur) * inv_dr, fmax(fabs(ut) * inv_rdt, fabs(uz + Ubase) * inv_dz)));
  }
  if (cfl) {  // warp max, then one atomic per warp (non-negative doubles order as integers)
    for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    const double cm = (double)cmax;
    if ((threadIdx.x & 31) == 0 && cm > 0.0)
      atomicMax((unsigned long long*)cfl, (unsigned long long)__double_as_longlong(cm));
  }
  __syncthreads();
  V* D = (C == A) ? B : A;
  const V* out;
  const int nfwd = kPackNz ? zc + (zc + 1) / 2 : 2 * zc;
  if constexpr (NTH > 0) out = block_fft_c<NTH, -1>(C, D, nfwd, ld, tw);
  else out = block_fft(C, D, nfwd, ld, pth, tw, -1);
  grid_dep_trigger_at(d, 2);
  for (int e = threadIdx.x; e < zc * M; e += blockDim.x) {
    const int m = e % M, zr = e / M, mc = m == 0 ? 0 : nth - m;
    const int rp = kPackNz ? zr : zr * 2;  // the (N_r + i N_theta) sequence of row zr
    const V y = out[rp * ld + m];
    const V yc = out[rp * ld + mc];
    const V nr = V{(T)0.5 * (y.x + yc.x), (T)0.5 * (y.y - yc.y)};
    const V nt = V{(T)0.5 * (y.y + yc.y), (T)-0.5 * (y.x - yc.x)};
    const long row = ((long)n * nz + z0 + zr) * M + m;
    ZN[row] = nr;
    ZN[fstride + row] = nt;
    if constexpr (kPackNz) {  // Z = F(a) + i F(b): F(a) = (Z + conj Z(-m)) / 2, F(b) = (Z - conj Z(-m)) / 2i
      const V w = out[(zc + (zr >> 1)) * ld + m], wc = out[(zc + (zr >> 1)) * ld + mc];
      ZN[2 * fstride + row] = (zr & 1) ? V{(T)0.5 * (w.y + wc.y), (T)-0.5 * (w.x - wc.x)}
                                       : V{(T)0.5 * (w.x + wc.x), (T)0.5 * (w.y - wc.y)};
    } else {
      ZN[2 * fstride + row] = out[(zr * 2 + 1) * ld + m];
    }
  }
}

size_t product_smem(const Dims& d, int zc, size_t vb) { return (2 * 3 * (size_t)zc * d.nth + d.nth) * vb; }

void launch_product32(const Dims& d, const DevSetup& s, const FftPlan& pth, const float2* Z6,
                      float2* ZN, cudaStream_t st) {
  dim3 g((d.nz + d.zc - 1) / d.zc, d.N, d.B);
  const size_t sm = product_smem(d, d.zc, sizeof(float2));
  with_fft_length(d.nth, [&](auto n) {
    launch_step_kernel(d, k_product<float2, decltype(n)::value>, g, dim3(transform_threads(g)), sm, st, d, pth,
                       (const float2*)s.tw_th32, Z6, ZN);
  });
}

void launch_product(const Dims& d, const DevSetup& s, const FftPlan& pth, const double2* Z6,
                    double2* ZN, cudaStream_t st) {
  dim3 g((d.nz + d.zc - 1) / d.zc, d.N, d.B);
  const size_t sm = product_smem(d, d.zc, sizeof(double2));
  with_fft_length(d.nth, [&](auto n) {
    launch_step_kernel(d, k_product<double2, decltype(n)::value>, g, dim3(transform_threads(g)), sm, st, d, pth,
                       (const double2*)s.tw_th, Z6, ZN);
  });
}

// ------------------------------------------------------------------ z analysis (A4)
template <typename V, int NZ>
__global__ void __launch_bounds__(256) k_zanalysis(Dims d, FftPlan pz, const V* __restrict__ twz,
                                                   const V* __restrict__ ZN, const double2* __restrict__ Nlin,
                                                   double2* __restrict__ Nout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nz = NZ > 0 ? NZ : d.nz, ld = nz + 1, M = d.M, K = d.K, nk = d.nk;
  const int MC = d.mca;
  V* A = (V*)smraw;
  V* B = A + 3 * MC * ld;
  V* tw = B + 3 * MC * ld;
  const int m0 = blockIdx.x * MC, n = blockIdx.y;
  const int mcn = min(MC, M - m0);
  twz = bofs(twz, d.ps);
  ZN = bofs(ZN, d.ss);
  Nlin = bofs(Nlin, d.ss);
  Nout = bofs(Nout, d.ss);
  const double Re = bofs(d.prm, d.ps)[kPrmRe];
  grid_dep_trigger_at(d, 1);
  for (int e = threadIdx.x; e < nz; e += blockDim.x) tw[e] = twz[e];
  const long fs = d.F;
  grid_dep_wait();
  // FP64 addends of an output point (linear terms, body force); a thread's
  // first point has them loaded before the transform, so that their latency
  // overlaps it
  auto addends = [&](long o, double2* ap, double2* am, double2* az) {
    *ap = *am = *az = double2{0.0, 0.0};
    if (d.forcing) {  // constant body force (shared by the trajectories of a group)
      *ap = d.forcing[o];
      *am = d.forcing[fs + o];
      *az = d.forcing[2 * fs + o];
    }
    if (Nlin) {  // terms linear in the perturbation, evaluated in FP64
      const double2 a = Nlin[o], b = Nlin[fs + o], c = Nlin[2 * fs + o];
      *ap = double2{ap->x + a.x, ap->y + a.y};
      *am = double2{am->x + b.x, am->y + b.y};
      *az = double2{az->x + c.x, az->y + c.y};
    }
  };
  auto out_index = [&](int e) {
    const int kk = e % nk, mc = e / nk;
    return ((long)(m0 + mc) * d.N + n) * nk + kk;
  };
  double2 pp, pm, pz0;
  const bool have0 = threadIdx.x < mcn * nk;
  if (have0 && (Nlin || d.forcing)) addends(out_index(threadIdx.x), &pp, &pm, &pz0);
  const long fstride = (long)d.N * nz * M;
  block_copy_batched<8, V>(
      3 * MC * nz,
      [&](int e) {
        const int mc = e % MC, z = (e / MC) % nz, f = e / (MC * nz);
        V v = V{0, 0};
        if (mc < mcn) v = ZN[f * fstride + ((long)n * nz + z) * M + m0 + mc];
        return v;
      },
      [&](int e, V v) {
        const int mc = e % MC, z = (e / MC) % nz, f = e / (MC * nz);
        A[(f * MC + mc) * ld + z] = v;
      });
  __syncthreads();
  const V* res;
  if constexpr (NZ > 0) res = block_fft_c<NZ, -1>(A, B, 3 * MC, ld, tw);
  else res = block_fft(A, B, 3 * MC, ld, pz, tw, -1);
  // scaling and the +- combination in the transform's precision, then FP64
  using T = typename Scalar<V>::T;
  const T sc = (T)d.inv_grid;
  grid_dep_trigger_at(d, 2);
  for (int e = threadIdx.x; e < mcn * nk; e += blockDim.x) {
    const int kk = e % nk, mc = e / nk, m = m0 + mc;
    const int k = kk - (K - 1);
    const int zp = k < 0 ? k + nz : k;
    const V r_ = res[(0 * MC + mc) * ld + zp], t_ = res[(1 * MC + mc) * ld + zp];
    const V z_ = res[(2 * MC + mc) * ld + zp];
    double2 np = double2{(double)(sc * (r_.x - t_.y)), (double)(sc * (r_.y + t_.x))};  // N+ = N_r + i N_theta
    double2 nm = double2{(double)(sc * (r_.x + t_.y)), (double)(sc * (r_.y - t_.x))};  // N- = N_r - i N_theta
    double2 nz2 = double2{(double)(sc * z_.x), (double)(sc * z_.y)};
    if (k == 0 && m == 0) nz2.x += 4.0 / Re;  // base driving force (laminar balance)
    const long o = ((long)m * d.N + n) * nk + kk;
    if (Nlin || d.forcing) {
      double2 ap, am, az;
      if (e == (int)threadIdx.x) {
        ap = pp;
        am = pm;
        az = pz0;
      } else {
        addends(o, &ap, &am, &az);
      }
      np.x += ap.x;
      np.y += ap.y;
      nm.x += am.x;
      nm.y += am.y;
      nz2.x += az.x;
      nz2.y += az.y;
    }
    Nout[o] = np;
    Nout[fs + o] = nm;
    Nout[2 * fs + o] = nz2;
  }
}

size_t zanalysis_smem(const Dims& d, int mc, size_t vb) {
  return (2 * 3 * (size_t)mc * (d.nz + 1) + d.nz) * vb;
}

void launch_zanalysis(const Dims& d, const DevSetup& s, const FftPlan& pz, const double2* ZN,
                      double2* Nout, cudaStream_t st) {
  dim3 g((d.M + d.mca - 1) / d.mca, d.N, d.B);
  const size_t sm = zanalysis_smem(d, d.mca, sizeof(double2));
  with_fft_length(d.nz, [&](auto n) {
    launch_step_kernel(d, k_zanalysis<double2, decltype(n)::value>, g, dim3(transform_threads(g)), sm, st, d, pz,
                       (const double2*)s.tw_z, ZN, (const double2*)nullptr, Nout);
  });
}

void launch_zanalysis32(const Dims& d, const DevSetup& s, const FftPlan& pz, const float2* ZN,
                        const double2* Nlin, double2* Nout, cudaStream_t st) {
  dim3 g((d.M + d.mca - 1) / d.mca, d.N, d.B);
  const size_t sm = zanalysis_smem(d, d.mca, sizeof(float2));
  with_fft_length(d.nz, [&](auto n) {
    launch_step_kernel(d, k_zanalysis<float2, decltype(n)::value>, g, dim3(transform_threads(g)), sm, st, d, pz,
                       (const float2*)s.tw_z32, ZN, Nlin, Nout);
  });
}

// ------------------------------------------------------------------ fused FP32 transforms (A2-A4)
// The mixed-precision nonlinear term after the curl, in one launch: a cluster
// of C blocks per (radial plane n, trajectory b) keeps the plane's
// half-physical fields in distributed shared memory instead of round trips
// through L2 between three kernels.
//   phase 1  block r takes m columns [r MC, (r+1) MC) of all six fields:
//            inverse z transforms (the z synthesis kernel's arithmetic);
//   phase 2  block r takes z rows [r ZR, (r+1) ZR): gathers those rows of
//            every m column from the blocks that own them, inverse theta
//            transforms, u x w (with the Coriolis term and the CFL maximum),
//            forward theta transforms (the product kernel's arithmetic);
//   phase 3  block r takes its m columns again: gathers them over all z rows,
//            forward z transforms, truncation, scaling, +- form and the FP64
//            addends (the z analysis kernel's arithmetic).
// Each transform runs the same block FFT on the same sequences as the
// three-kernel path, so the results are identical to it.
namespace cg = cooperative_groups;

__host__ __device__ inline int fused_mc(int M, int C) { return (M + C - 1) / C; }
__host__ __device__ inline int fused_zr(int nz, int C) { return (nz + C - 1) / C; }

size_t fused32_smem(const Dims& d, int C) {
  const int MC = fused_mc(d.M, C), ZR = fused_zr(d.nz, C);
  return (2 * 6 * (size_t)MC * (d.nz + 1) + 3 * (size_t)ZR * d.M + d.nz + d.nth) * sizeof(float2);
}

template <int NZ, int NTH>
__global__ void __launch_bounds__(256) k_nl_fused32(Dims d, int C, const float2* __restrict__ twz,
                                                    const float2* __restrict__ twth,
                                                    const float2* __restrict__ W6,
                                                    const double2* __restrict__ Nlin,
                                                    double2* __restrict__ Nout) {
  using V = float2;
  using T = float;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LDZ = NZ + 1;
  const int M = d.M, K = d.K, nk = d.nk, N = d.N;
  const int MC = fused_mc(M, C), ZR = fused_zr(NZ, C);
  const int rank = (int)cl.block_rank();
  const int n = blockIdx.x / C;
  V* A = (V*)smraw;            // [6 MC][LDZ]  phase 1 (then phase 3)
  V* B = A + 6 * MC * LDZ;     // [6 MC][LDZ]  phase 1 ping-pong (then phase 2)
  V* ZNl = B + 6 * MC * LDZ;   // [3][ZR][M]   product spectra of this block's z rows
  V* tz = ZNl + 3 * ZR * M;    // [NZ]
  V* tth = tz + NZ;            // [NTH]
  twz = bofs(twz, d.ps);
  twth = bofs(twth, d.ps);
  W6 = bofs(W6, d.ss);
  Nlin = bofs(Nlin, d.ss);
  Nout = bofs(Nout, d.ss);
  const double Re = bofs(d.prm, d.ps)[kPrmRe];
  for (int e = threadIdx.x; e < NZ; e += blockDim.x) tz[e] = twz[e];
  for (int e = threadIdx.x; e < NTH; e += blockDim.x) tth[e] = twth[e];
  const long fs = d.F;
  const int m0 = rank * MC;
  const int mcn = max(0, min(MC, M - m0));

  // ---- phase 1: inverse z transforms of this block's m columns, six fields
  for (int e = threadIdx.x; e < 6 * MC * NZ; e += blockDim.x) {
    const int z = e % NZ, col = e / NZ, f = col / MC, mc = col % MC;
    const int k = z < K ? z : z - NZ;
    V v = V{0, 0};
    if (mc < mcn && (z < K || z > NZ - K)) v = W6[f * fs + ((long)(m0 + mc) * N + n) * nk + k + K - 1];
    A[col * LDZ + z] = v;
  }
  __syncthreads();
  V* res1 = block_fft_c<NZ, +1, true>(A, B, 6 * MC, LDZ, tz);
  V* free1 = (res1 == A) ? B : A;
  cl.sync();  // every block's half-physical columns are in place

  // ---- phase 2: this block's z rows: theta transforms and the product
  const int z0 = rank * ZR;
  const int zrn = max(0, min(ZR, NZ - z0));
  const int ZC = max(1, min(max(zrn, 1), (6 * MC * LDZ) / (6 * NTH)));
  V* P0 = free1;               // [3 ZC][NTH]
  V* P1 = free1 + 3 * ZC * NTH;  // [3 ZC][NTH]
  double* cfl = bofs(d.cfl, d.ss);
  T inv_dr = 0, inv_rdt = 0, inv_dz = 0, Ubase = 0;
  if (cfl) {
    const double* rinv = bofs(d.rinv_cfl, d.ps);
    const T one = 1, rn = one / (T)rinv[n];
    const T rm = n > 0 ? one / (T)rinv[n - 1] : -rn;
    const T rp = n < N - 1 ? one / (T)rinv[n + 1] : one + (one - rm);
    const T twopi = (T)6.283185307179586;
    inv_dr = one / fmin(rn - rm, rp - rn);
    inv_rdt = (T)(d.m_p * NTH) / (twopi * rn);
    inv_dz = (T)d.alpha * (T)NZ / twopi;
    Ubase = one - rn * rn;
  }
  T cmax = 0;
  for (int c0 = 0; c0 < zrn; c0 += ZC) {
    const int zc = min(ZC, zrn - c0);
    // spectra of the pairs (u_r,u_t), (u_z,w_r), (w_t,w_z):  Z = A + i B
    for (int e = threadIdx.x; e < zc * 3 * NTH; e += blockDim.x) {
      const int q = e % NTH, pr = (e / NTH) % 3, zr = e / (3 * NTH);
      const int z = z0 + c0 + zr;
      V v = V{0, 0};
      const int mq = q < M ? q : (q > NTH - M ? NTH - q : -1);
      if (mq >= 0) {
        const V* src = cl.map_shared_rank(res1, mq / MC);
        V a = src[((2 * pr) * MC + mq % MC) * LDZ + z], b = src[((2 * pr + 1) * MC + mq % MC) * LDZ + z];
        if (q < M) {
          if (q == 0) {
            a.y = 0;
            b.y = 0;
          }
          v = V{a.x - b.y, a.y + b.x};
        } else {
          v = V{a.x + b.y, -a.y + b.x};  // conj(a) + i conj(b)
        }
      }
      P0[(zr * 3 + pr) * NTH + q] = v;
    }
    __syncthreads();
    V* res = block_fft_c<NTH, +1, true>(P0, P1, 3 * zc, NTH, tth);
    V* Cb = (res == P0) ? P1 : P0;
    for (int e = threadIdx.x; e < zc * NTH; e += blockDim.x) {
      const int q = e % NTH, zr = e / NTH;
      const V x0 = res[(zr * 3 + 0) * NTH + q], x1 = res[(zr * 3 + 1) * NTH + q], x2 = res[(zr * 3 + 2) * NTH + q];
      const T ur = x0.x, ut = x0.y, uz = x1.x, wr = x1.y, wt = x2.x, wz = x2.y;
      T nr = ut * wz - uz * wt, nt = uz * wr - ur * wz, nz = ur * wt - ut * wr;
      if (d.rotate) {  // Coriolis -2 Omega x u, Omega in cylindrical components at theta_q
        T sn, cs;
        sincos_pi((T)(2 * q) / (T)(d.m_p * NTH), &sn, &cs);
        const T rx = (T)d.rot_x, ry = (T)d.rot_y;
        const T o_r = rx * cs + ry * sn, o_t = -rx * sn + ry * cs;
        const T o_z = (T)d.rot_z;
        nr -= (T)2 * (o_t * uz - o_z * ut);
        nt -= (T)2 * (o_z * ur - o_r * uz);
        nz -= (T)2 * (o_r * ut - o_t * ur);
      }
      Cb[(zr * 2 + 0) * NTH + q] = V{nr, nt};
      Cb[(zr * 2 + 1) * NTH + q] = V{nz, (T)0};
      if (cfl) cmax = fmax(cmax, fmax(fabs(ur) * inv_dr, fmax(fabs(ut) * inv_rdt, fabs(uz + Ubase) * inv_dz)));
    }
    __syncthreads();
    V* Db = (Cb == P0) ? P1 : P0;
    const V* out = block_fft_c<NTH, -1>(Cb, Db, 2 * zc, NTH, tth);
    for (int e = threadIdx.x; e < zc * M; e += blockDim.x) {
      const int m = e % M, zr = e / M;
      const V y = out[(zr * 2 + 0) * NTH + m];
      const V yc = out[(zr * 2 + 0) * NTH + (m == 0 ? 0 : NTH - m)];
      const int row = c0 + zr;
      ZNl[(0 * ZR + row) * M + m] = V{(T)0.5 * (y.x + yc.x), (T)0.5 * (y.y - yc.y)};
      ZNl[(1 * ZR + row) * M + m] = V{(T)0.5 * (y.y + yc.y), (T)-0.5 * (y.x - yc.x)};
      ZNl[(2 * ZR + row) * M + m] = out[(zr * 2 + 1) * NTH + m];
    }
    __syncthreads();  // P0 / P1 are reused by the next chunk of rows
  }
  if (cfl) {  // warp max, then one atomic per warp (non-negative doubles order as integers)
    for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    const double cm = (double)cmax;
    if ((threadIdx.x & 31) == 0 && cm > 0.0)
      atomicMax((unsigned long long*)cfl, (unsigned long long)__double_as_longlong(cm));
  }
  cl.sync();  // every block's product spectra are in place; nobody reads res1 any more

  // ---- phase 3: forward z transforms of this block's m columns, three fields
  V* A3 = A;
  V* B3 = A + 3 * MC * LDZ;
  for (int e = threadIdx.x; e < 3 * MC * NZ; e += blockDim.x) {
    const int z = e % NZ, col = e / NZ, f = col / MC, mc = col % MC;
    V v = V{0, 0};
    if (mc < mcn) {
      const V* src = cl.map_shared_rank(ZNl, z / ZR);
      v = src[(f * ZR + z % ZR) * M + m0 + mc];
    }
    A3[col * LDZ + z] = v;
  }
  cl.sync();  // every remote read is done before any block moves on or exits
  const V* res3 = block_fft_c<NZ, -1>(A3, B3, 3 * MC, LDZ, tz);
  const T sc = (T)d.inv_grid;
  for (int e = threadIdx.x; e < mcn * nk; e += blockDim.x) {
    const int kk = e % nk, mc = e / nk, m = m0 + mc;
    const int k = kk - (K - 1);
    const int zp = k < 0 ? k + NZ : k;
    const V r_ = res3[(0 * MC + mc) * LDZ + zp], t_ = res3[(1 * MC + mc) * LDZ + zp];
    const V z_ = res3[(2 * MC + mc) * LDZ + zp];
    double2 np = double2{(double)(sc * (r_.x - t_.y)), (double)(sc * (r_.y + t_.x))};  // N+ = N_r + i N_theta
    double2 nm = double2{(double)(sc * (r_.x + t_.y)), (double)(sc * (r_.y - t_.x))};  // N- = N_r - i N_theta
    double2 nz2 = double2{(double)(sc * z_.x), (double)(sc * z_.y)};
    if (k == 0 && m == 0) nz2.x += 4.0 / Re;  // base driving force (laminar balance)
    const long o = ((long)m * N + n) * nk + kk;
    double2 ap = double2{0.0, 0.0}, am = ap, az = ap;
    if (d.forcing) {  // constant body force (shared by the trajectories of a group)
      ap = d.forcing[o];
      am = d.forcing[fs + o];
      az = d.forcing[2 * fs + o];
    }
    if (Nlin) {  // terms linear in the perturbation, evaluated in FP64
      const double2 a = Nlin[o], b = Nlin[fs + o], c = Nlin[2 * fs + o];
      ap = double2{ap.x + a.x, ap.y + a.y};
      am = double2{am.x + b.x, am.y + b.y};
      az = double2{az.x + c.x, az.y + c.y};
    }
    if (Nlin || d.forcing) {
      np.x += ap.x;
      np.y += ap.y;
      nm.x += am.x;
      nm.y += am.y;
      nz2.x += az.x;
      nz2.y += az.y;
    }
    Nout[o] = np;
    Nout[fs + o] = nm;
    Nout[2 * fs + o] = nz2;
  }
}

// Cluster size for a fused launch of this shape (0: the shape takes the
// three-kernel path): transform lengths with a compiled plan up to 96;
// d.fused = 2, 4 or 8 forces the cluster size, 1 chooses it (eight blocks
// per plane when the grid would otherwise leave SMs idle, else four).
int fused32_cluster(const Dims& d) {
  auto ok = [](int n) { return n == 48 || n == 72 || n == 96; };
  if (!d.fused || !ok(d.nz) || !ok(d.nth)) return 0;
  int dev = 0, sms = 152, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int C = d.fused >= 2 ? d.fused : ((long)4 * d.N * d.B < 2L * sms ? 8 : 4);
  if (fused32_smem(d, C) > (size_t)optin) return 0;
  if ((long)fused_mc(d.M, C) * (d.nz + 1) < d.nth) return 0;  // phase 2 needs one row's buffers
  return C;
}

template <int NZ, int NTH>
void launch_fused_len(const Dims& d, const DevSetup& s, int C, const float2* W6, const double2* Nlin,
                      double2* Nout, cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C * d.N, 1, d.B);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = fused32_smem(d, C);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_nl_fused32<NZ, NTH>, d, C, (const float2*)s.tw_z32, (const float2*)s.tw_th32, W6,
                     Nlin, Nout);
}

template <class F>
void with_fused_lengths(int nz, int nth, F&& f) {
  auto inner = [&](auto z) {
    switch (nth) {
      case 48: f(z, std::integral_constant<int, 48>{}); break;
      case 72: f(z, std::integral_constant<int, 72>{}); break;
      default: f(z, std::integral_constant<int, 96>{}); break;
    }
  };
  switch (nz) {
    case 48: inner(std::integral_constant<int, 48>{}); break;
    case 72: inner(std::integral_constant<int, 72>{}); break;
    default: inner(std::integral_constant<int, 96>{}); break;
  }
}

bool launch_nl_fused32(const Dims& d, const DevSetup& s, const float2* W6, const double2* Nlin, double2* Nout,
                       cudaStream_t st) {
  const int C = fused32_cluster(d);
  if (!C) return false;
  with_fused_lengths(d.nz, d.nth, [&](auto z, auto t) {
    launch_fused_len<decltype(z)::value, decltype(t)::value>(d, s, C, W6, Nlin, Nout, st);
  });
  return true;
}

// ------------------------------------------------------------------ linear solve (A5-A7)
struct SolveDev {
  const double* d1;
  const double* rinv;
  const double* wq;
  const int* hop;
  const double* luH;
  const double* luP;
  const double* basis;
  const double2* ainv;
  const double* G;
  const double* prm;
  int nJ;
  int stage;  // u_j and the influence responses staged in shared memory
  const float* d1f;
  const double* r;
  // split solve: both blocks' factors, spikes, interface inverses
  const double* luH2;
  const double* luP2;
  const double* spkH;
  const double* spkP;
  const double* rH;
  const double* rP;
};

// Bulk L2 prefetch by the TMA unit: p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Asynchronous global -> shared copies (8 or 16 bytes, both addresses aligned
// to the size); completion by commit groups, visibility by a block barrier.
__device__ __forceinline__ void cp_async8(void* sm, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(sm)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* sm, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(sm)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int G>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(G) : "memory"); }

// Shared memory of a solve block: the working arrays, then (when they fit in
// ~100 KB, i.e. for moderate N) u_j and the influence responses of the tile,
// staged by asynchronous copies at the start so that the right-hand sides,
// the influence step and the write-out read them from shared memory.
// The host stages only where that costs no resident blocks (see
// launch_solve); the launch gives the staged size then, the base size else.
// Rows of P: the pressure, later the influence step's scratch (12 complex per mode).
__host__ __device__ constexpr int solve_prows(int N) { return N > 12 ? N : 12; }
// sp: the split solve's interface values (6T chains x 8 doubles) after misc.
__host__ __device__ constexpr size_t solve_smem_base(int N, int T, bool sp = false) {
  return (size_t)(N * T + solve_prows(N) * T + 4 * T) * 16 + (size_t)6 * N * T * 8 +
         (size_t)(2 * N * 9 + 3 * N + 2) * 8 + 16 + (sp ? (size_t)48 * T * 8 : 0);
}
__host__ __device__ constexpr size_t solve_smem_staged(int N, int T, bool sp = false) {
  return solve_smem_base(N, T, sp) + (size_t)96 * N * T;
}
// The FP32 copy of u_theta for the mixed-precision curl of the solved state.
__host__ __device__ constexpr size_t solve_smem_curl32(int N, int T) { return (size_t)8 * N * T; }
__host__ __device__ constexpr bool solve_stage_fits(int N, int T) { return solve_smem_staged(N, T) <= 100 * 1024; }

// Banded substitution on one real right-hand side held in shared memory at
// x[i * st], i < N, by a group of 4 consecutive lanes (column-oriented):
// lane t keeps the partial sum of row c+1+t (and of row c+5+t for the wall
// rows, whose lower band reaches 8); once row c is final its value is
// broadcast and each lane subtracts its row's multiple of it.  The factor is
// stored by columns (13 N values, see to_columns on the host): [N][4]
// L(c+1+t, c), [N][4] L(c+5+t, c), [N] 1/U_ii, [N][4] U(c-1-t, c) / U_ii,
// zeros outside the band, so the four lanes of a chain read one 32-byte run
// per column.  Each lane needs one factor entry per row; it is loaded kAhead
// rows ahead into a register queue (the loop is unrolled by kAhead so the
// queue is indexed statically), which keeps the L2 latency off the recursion.
// All 32 lanes of the warp must call this together (8 right-hand sides per
// warp).
__device__ __forceinline__ void band_solve4(const double* __restrict__ L, double* x, int st, int N) {
  const int t = threadIdx.x & 3;
  const unsigned full = 0xffffffffu;
  constexpr int kAhead = 16;
  const double* Lw = L + 4 * N;  // L(c+5+t, c)
  const double* Dg = L + 8 * N;  // 1/U_ii
  const double* Uc = L + 9 * N;  // U(c-1-t, c) / U_(c-1-t)
  // forward: y = L^{-1} b.  Row c+1+t's entry in column c, queued kAhead rows
  // ahead; on the wall rows (c >= N-9) also row c+5+t's entry in column c,
  // all nine loaded up front.
  auto la_of = [&](int c) { return c < N ? __ldg(L + c * 4 + t) : 0.0; };
  double qa[kAhead], qw[9];
#pragma unroll
  for (int j = 0; j < kAhead; ++j) qa[j] = la_of(j);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int c = N - 9 + j;
    qw[j] = c >= 0 ? __ldg(Lw + c * 4 + t) : 0.0;
  }
  double sa = t < N ? x[t * st] : 0.0;
  double sb = 4 + t < N ? x[(4 + t) * st] : 0.0;
  for (int c0 = 0; c0 < N; c0 += kAhead) {
#pragma unroll
    for (int j = 0; j < kAhead; ++j) {
      const int c = c0 + j;  // warp-uniform
      if (c < N) {
        const double y = __shfl_sync(full, sa, 0, 4);
        if (t == 0) x[c * st] = y;
        const double next_b = (t == 3 && c + 8 < N) ? x[(c + 8) * st] : 0.0;
        double san = __shfl_down_sync(full, sa, 1, 4);
        const double sb0 = __shfl_sync(full, sb, 0, 4);
        double sbn = __shfl_down_sync(full, sb, 1, 4);
        if (t == 3) {
          san = sb0;
          sbn = next_b;
        }
        sa = san - qa[j] * y;
        if (c >= N - 9) {
          double w = qw[0];
#pragma unroll
          for (int q = 1; q < 9; ++q)
            if (c == N - 9 + q) w = qw[q];
          sbn -= w * y;
        }
        sb = sbn;
        qa[j] = la_of(c + kAhead);
      }
    }
  }
  // y_i / U_ii for all rows at once (off the recursion; the U rows are stored
  // scaled by 1/U_ii, so the backward sweep has a single FMA per row)
  __syncwarp();
  for (int i = t; i < N; i += 4) x[i * st] *= __ldg(Dg + i);
  __syncwarp();
  // backward: x = U~^{-1} (y / diag U).  Row c-1-t's scaled entry in column c.
  auto ua_of = [&](int c) { return c >= 0 ? __ldg(Uc + c * 4 + t) : 0.0; };
  double qu[kAhead];
#pragma unroll
  for (int j = 0; j < kAhead; ++j) qu[j] = ua_of(N - 1 - j);
  sa = N - 1 - t >= 0 ? x[(N - 1 - t) * st] : 0.0;
  for (int c0 = N - 1; c0 >= 0; c0 -= kAhead) {
#pragma unroll
    for (int j = 0; j < kAhead; ++j) {
      const int c = c0 - j;  // warp-uniform
      if (c >= 0) {
        const double xc = __shfl_sync(full, sa, 0, 4);
        if (t == 0) x[c * st] = xc;
        const double next_y = (t == 3 && c - 4 >= 0) ? x[(c - 4) * st] : 0.0;
        double san = __shfl_down_sync(full, sa, 1, 4);
        if (t == 3) san = next_y;
        sa = san - qu[j] * xc;
        qu[j] = ua_of(c - kAhead);
      }
    }
  }
}

// One block: T consecutive k at fixed m (24T threads).  Row-parallel phases
// use all threads over (chain, row); only the banded substitutions are
// sequential in r, with 4 lanes per real right-hand side (2T pressure chains,
// then 6T velocity chains = (u+, u-, u_z) x T modes x (re, im)).  While warp
// 0 solves the pressure system the other warps assemble the p-independent part
// of the velocity right-hand sides (and stage u_j and the influence
// responses); the last pass applies u_j, the influence correction and the
// flux correction on the way out to global memory, and with a.curl the block
// then takes the curl of its new state for the next nonlinear evaluation.
//
// Resident blocks per SM the register budget must allow (the shared-memory
// footprints of the tiles allow about as many at moderate N).
template <int T, bool SP>
constexpr int solve_min_blocks() {
  return SP ? 3 : (T == 4 ? 4 : (T == 8 ? 3 : 2));
}

// Interface and correction of the split solve for nch chains held in x
// (chain c's column at x + col(c), rows at stride st) after both halves were
// substituted: z = R (y_T[k-4:k], y_B[0:4]) per chain, then every row
// x_i -= S_i . z_B (top half) or S_i . z_T (bottom half), k = N/2.  spk: per
// operator N rows of 4; R: per operator 8 x 8.  Ends with a block barrier.
template <int NB, typename OpOf>
__device__ __forceinline__ void spike_fix(int tid, int N, int nch, int st, double* x, const double* __restrict__ spk,
                                          const double* __restrict__ R, double* Zs, OpOf op_of) {
  const int kh = N >> 1;
  for (int e = tid; e < nch * 8; e += NB) {
    const int c = e >> 3, q = e & 7;
    const double* Rc = R + (long)op_of(c) * 64 + q * 8;
    const double* xc = x + c;
    double z = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) z = fma(Rc[b], xc[(kh - 4 + b) * st], z);
#pragma unroll
    for (int b = 0; b < 4; ++b) z = fma(Rc[4 + b], xc[(kh + b) * st], z);
    Zs[e] = z;
  }
  __syncthreads();
  for (int e = tid; e < nch * N; e += NB) {
    const int c = e % nch, i = e / nch;
    const double* S = spk + ((long)op_of(c) * N + i) * 4;
    const double* z = Zs + c * 8 + (i < kh ? 4 : 0);
    double v = x[i * st + c];
#pragma unroll
    for (int q = 0; q < 4; ++q) v = fma(-S[q], z[q], v);
    x[i * st + c] = v;
  }
  __syncthreads();
}

// SP: the split (two-partition) solve for the latency-bound grids -- each
// chain's substitution runs on 8 lanes, the two halves of its rows at once
// (twice the threads; the other phases use them too).
template <int T, bool SP = false>
__global__ void __launch_bounds__((SP ? 48 : 24) * T, solve_min_blocks<T, SP>())
    k_solve(Dims d, SolveDev s, SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = d.N, nk = d.nk, M = d.M, K = d.K;
  constexpr int NT = 6 * T;                // velocity right-hand sides (chains)
  constexpr int NB = (SP ? 48 : 24) * T;   // threads: 4 (SP: 8) lanes per velocity chain
  constexpr int NP = (SP ? 16 : 8) * T;    // threads of the pressure substitution (2T chains)
  // X holds N_eff first (chain layout: field f, mode mi, re/im part), then
  // the velocity right-hand sides built on it in place, then the chains'
  // solutions; S and P are reused by the influence step and the curl.
  double2* S = (double2*)smraw;                // [N][T]     N+ + N- (later u_j near the wall, u_r)
  double2* P = S + N * T;                      // [N][T]     pressure (later influence scratch, u_theta)
  double2* coef = P + solve_prows(N) * T;      // [T][4]     influence coefficients
  double* X = (double*)(coef + 4 * T);         // [N][6T]    N_eff -> right-hand sides -> velocity chains
  double* W1 = X + N * NT;                     // [2][N][9]  first-derivative stencils
  double* RI = W1 + 2 * N * 9;                 // [N]        1/r
  double* RIp = RI + N;                        // [N]        (1 + m~) / (2r)
  double* RIm = RIp + N;                       // [N]        (1 - m~) / (2r)
  double* misc = RIm + N;                      // [2]        flux correction
  const bool stage = s.stage;
  // u_j near the wall for the influence step, when not staged: in S (free
  // after the pressure right-hand side) if it holds [T][19], else from global
  double2* UW = S;
  const bool uw_in_s = !stage && N >= 19;
  double* Zs = misc + 2;                       // [6T][8]    split-solve interface values (SP)
  double2* UJ = (double2*)(((size_t)(Zs + (SP ? 48 * T : 0)) + 15) & ~(size_t)15);  // [3][N][T] u_j (stage)
  double* BS = (double*)(UJ + 3 * N * T);                             // [T][6N]   responses (stage)
  float2* UT32 = stage ? (float2*)(BS + 6 * N * T) : (float2*)UJ;     // [N][T] FP32 u_theta (curl 2)
  // N_eff of field f, row i, mode mi as a complex pair in X's chain layout
  auto ne_at = [&](int f, int i, int mi) -> double2& {
    return *(double2*)(X + (long)i * NT + ((f * T + mi) << 1));
  };
  const int m = blockIdx.y, kk0 = blockIdx.x * T, tid = threadIdx.x;
  const int mt = d.m_p * m, ps = mt & 1, pv = ps ^ 1;
  s.d1 = bofs(s.d1, d.ps);
  s.rinv = bofs(s.rinv, d.ps);
  s.wq = bofs(s.wq, d.ps);
  s.hop = bofs(s.hop, d.ps);
  s.luH = bofs(s.luH, d.ps);
  s.luP = bofs(s.luP, d.ps);
  s.basis = bofs(s.basis, d.ps);
  s.ainv = bofs(s.ainv, d.ps);
  s.G = bofs(s.G, d.ps);
  s.prm = bofs(s.prm, d.ps);
  s.d1f = bofs(s.d1f, d.ps);
  s.r = bofs(s.r, d.ps);
  if constexpr (SP) {
    s.luH2 = bofs(s.luH2, d.ps);
    s.luP2 = bofs(s.luP2, d.ps);
    s.spkH = bofs(s.spkH, d.ps);
    s.spkP = bofs(s.spkP, d.ps);
    s.rH = bofs(s.rH, d.ps);
    s.rP = bofs(s.rP, d.ps);
  }
  a.W6 = bofs(a.W6, d.ss);
  a.Nlin = bofs(a.Nlin, d.ss);
  a.Uj = bofs(a.Uj, d.ss);
  a.Na = bofs(a.Na, d.ss);
  a.Nb = bofs(a.Nb, d.ss);
  a.Uout = bofs(a.Uout, d.ss);
  a.beta_p = bofs(a.beta_p, d.ss);
  const double ci = s.prm[kPrmCi], cu = s.prm[kPrmCu];  // 1 / (c dt), (1 - c) / c
  const long fs = d.F;
  const long base = (long)m * N * nk;
  const double* wv = W1 + pv * N * 9;  // stencils of u_r, u_theta parity
  const double* ws = W1 + ps * N * 9;  // stencils of u_z, p parity
  // chain c -> (field f, mode mi, part); element (f, row i, mode mi) of a field
  auto uj = [&](int f, int i, int mi) {
    return a.Uj[f * fs + base + (long)i * nk + min(kk0 + mi, nk - 1)];
  };

  grid_dep_trigger_at(d, 1);
  // Pull this block's factor blocks (pressure, u+, u-, u_z per mode) and
  // basis blocks towards L2 with one bulk prefetch each, so they arrive while
  // the right-hand sides are assembled.  Factor blocks start on 16 bytes only
  // for even N (104 N bytes per operator); basis blocks (48 N bytes) always do.
  if (tid < 5 * T) {
    const int mi = tid % T, which = tid / T;
    const int ik = abs(min(kk0 + mi, nk - 1) - (K - 1));
    if (which == 4) {
      if (!stage) prefetch_l2_bulk(s.basis + (long)(ik * M + m) * 6 * N, 48u * N);
    } else if (!(N & 1)) {
      const long op = which == 0 ? ((ik == 0 && m == 0) ? K * M : ik * M + m) : ik * s.nJ + s.hop[3 * m + which - 1];
      prefetch_l2_bulk((which == 0 ? (SP ? s.luP2 : s.luP) : (SP ? s.luH2 : s.luH)) + op * N * kLuSlots,
                       (unsigned)N * kLuSlots * 8u);
    }
  }

  // The stencils by asynchronous copies, waited for at the first barrier.
  for (int e = tid; e < 2 * N * 9; e += NB) cp_async8(W1 + e, s.d1 + e);
  cp_async_commit();

  // ---- N_eff = wa N_a + wb N_b, and N+ + N- for the divergence
  for (int e = tid; e < N; e += NB) {
    const double ri = s.rinv[e];
    RI[e] = ri;
    RIp[e] = 0.5 * (1 + mt) * ri;
    RIm[e] = 0.5 * (1 - mt) * ri;
  }
  grid_dep_wait();  // everything above read setup data only
#pragma unroll 4
  for (int e = tid; e < 3 * N * T; e += NB) {
    const int mi = e % T, i = (e / T) % N, f = e / (T * N);
    const long g = f * fs + base + (long)i * nk + min(kk0 + mi, nk - 1);
    const double2 u = a.Na[g];
    double2 v = u;
    if (a.wa != 1.0) v = double2{a.wa * u.x, a.wa * u.y};  // (the predictor takes N_a as it is)
    if (a.Nb) {
      const double2 w = a.Nb[g];
      v.x += a.wb * w.x;
      v.y += a.wb * w.y;
    }
    ne_at(f, i, mi) = v;
  }
  cp_async_wait<0>();
  __syncthreads();
  for (int e = tid; e < N * T; e += NB) {
    const int mi = e % T, i = e / T;
    const double2 p = ne_at(0, i, mi), q = ne_at(1, i, mi);
    S[e] = double2{p.x + q.x, p.y + q.y};
  }
  __syncthreads();

  // Row-parallel phases over (mode, row) give each thread one fixed mode
  // mi_t = tid % T and the rows tid / T, tid / T + NB / T, ...
  const int mi_t = tid % T;
  const double ak_t = d.alpha * (min(kk0 + mi_t, nk - 1) - (K - 1));

  // ---- pressure right-hand side: div N_eff (rows < N-1), 0 at the wall
  for (int i = tid / T; i < N; i += NB / T) {
    double2 b = double2{0.0, 0.0};
    if (i < N - 1) {
      const int lo = row_lo_d(i, N);
      double ax = 0.0, ay = 0.0;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const double2 sv = S[(lo + q) * T + mi_t];
        const double w = wv[i * 9 + q];
        ax = fma(w, sv.x, ax);
        ay = fma(w, sv.y, ay);
      }
      const double2 np = ne_at(0, i, mi_t), nm = ne_at(1, i, mi_t), nz = ne_at(2, i, mi_t);
      b.x = fma(0.5, ax, fma(RIp[i], np.x, fma(RIm[i], nm.x, -ak_t * nz.y)));
      b.y = fma(0.5, ay, fma(RIp[i], np.y, fma(RIm[i], nm.y, ak_t * nz.x)));
    }
    P[i * T + mi_t] = b;
  }
  __syncthreads();

  if (tid < NP) {
    // ---- pressure-Poisson solve (provisional dp/dr(1) = 0; (0,0): p(1) = 0)
    const int j = tid >> (SP ? 3 : 2), part = j & 1, mi = j >> 1;
    const int k = min(kk0 + mi, nk - 1) - (K - 1), ik = abs(k);
    const int op = (ik == 0 && m == 0) ? K * M : ik * M + m;
    if constexpr (SP) {  // lanes 0-3 of the chain's 8: top half, 4-7: bottom half
      const int h = (tid >> 2) & 1, kh = N >> 1;
      band_solve4(s.luP2 + ((long)op * N + h * kh) * kLuSlots, (double*)P + 2 * mi + part + h * kh * 2 * T, 2 * T,
                  kh);
    } else {
      band_solve4(s.luP + (long)op * N * kLuSlots, (double*)P + 2 * mi + part, 2 * T, N);
    }
  } else {
    // ---- meanwhile: the p-independent part of the velocity right-hand sides
    for (int e = tid - NP; e < N * NT; e += NB - NP) {
      const int c = e % NT, i = e / NT;
      const int part = c & 1, mi = (c >> 1) % T, f = (c >> 1) / T;
      double b = 0.0;
      if (i < N - 1) {
        const double2 u = uj(f, i, mi);
        if (stage && part == 0) UJ[(f * N + i) * T + mi] = u;
        b = fma(ci, part ? u.y : u.x, X[i * NT + c]);  // X held N_eff of this chain's element
      }
      X[i * NT + c] = b;
    }
    // u_j near the wall and the inverse influence matrices of the tile, for
    // the influence step (rows N-9..N-1 of u+, u-; row N-1 of u_z)
    // (staged: u_j of the wall row and the influence responses of the tile
    // into shared memory instead, for the influence step and the write-out)
    if (stage) {
      for (int e = tid - NP; e < 3 * T; e += NB - NP) {
        const int mi = e % T, f = e / T;
        UJ[(f * N + N - 1) * T + mi] = uj(f, N - 1, mi);
      }
      for (int e = tid - NP; e < 3 * N * T; e += NB - NP) {  // 16-byte chunks, 3N per mode
        const int mi = e / (3 * N), ch = e % (3 * N);
        const int ik = abs(min(kk0 + mi, nk - 1) - (K - 1));
        cp_async16(BS + (long)mi * 6 * N + 2 * ch, s.basis + (long)(ik * M + m) * 6 * N + 2 * ch);
      }
      cp_async_commit();
      cp_async_wait<0>();
    }
    if (uw_in_s) {
      for (int e = tid - NP; e < 19 * T; e += NB - NP) {
        const int mi = e % T, w = e / T;
        const int f = w < 18 ? w / 9 : 2, i = w < 18 ? N - 9 + w % 9 : N - 1;
        UW[mi * 19 + w] = uj(f, i, mi);
      }
    }
  }
  __syncthreads();
  if constexpr (SP)  // the pressure chains' interface and correction
    spike_fix<NB>(tid, N, 2 * T, 2 * T, (double*)P, s.spkP, s.rP, Zs, [&](int c) {
      const int ik = abs(min(kk0 + (c >> 1), nk - 1) - (K - 1));
      return (ik == 0 && m == 0) ? K * M : ik * M + m;
    });

  // ---- d_r p per (mode, row), subtracted at once from the right-hand sides of
  //      the three fields (rows < N-1):
  //      (grad p)+- = d_r p -+ m~ p / r,  (grad p)_z = i ak p
  for (int i = tid / T; i < N - 1; i += NB / T) {
    const int lo = row_lo_d(i, N);
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const double2 pv2 = P[(lo + q) * T + mi_t];
      const double w = ws[i * 9 + q];
      ax = fma(w, pv2.x, ax);
      ay = fma(w, pv2.y, ay);
    }
    const double2 pp = P[i * T + mi_t];
    const double mr = mt * RI[i];
    double* xr = X + i * NT;
    const int c0 = mi_t << 1, c1 = (T + mi_t) << 1, c2 = (2 * T + mi_t) << 1;
    xr[c0] = fma(mr, pp.x, xr[c0] - ax);
    xr[c0 + 1] = fma(mr, pp.y, xr[c0 + 1] - ay);
    xr[c1] = fma(-mr, pp.x, xr[c1] - ax);
    xr[c1 + 1] = fma(-mr, pp.y, xr[c1 + 1] - ay);
    xr[c2] = fma(ak_t, pp.y, xr[c2]);
    xr[c2 + 1] = fma(-ak_t, pp.x, xr[c2 + 1]);
  }
  __syncthreads();

  // ---- implicit viscous solves (1/dt - cL) v = rhs, Dirichlet 0
  {  // 6T chains x 4 (SP: 8) lanes = all threads
    const int c = tid >> (SP ? 3 : 2);
    const int mi = (c >> 1) % T, f = (c >> 1) / T;
    const int k = min(kk0 + mi, nk - 1) - (K - 1), ik = abs(k);
    const int op = ik * s.nJ + s.hop[3 * m + f];
    if constexpr (SP) {
      const int h = (tid >> 2) & 1, kh = N >> 1;
      band_solve4(s.luH2 + ((long)op * N + h * kh) * kLuSlots, X + c + h * kh * NT, NT, kh);
    } else {
      band_solve4(s.luH + (long)op * N * kLuSlots, X + c, NT, N);
    }
  }
  __syncthreads();
  if constexpr (SP)  // the velocity chains' interface and correction
    spike_fix<NB>(tid, N, NT, NT, X, s.spkH, s.rH, Zs, [&](int c) {
      const int ik = abs(min(kk0 + ((c >> 1) % T), nk - 1) - (K - 1));
      return ik * s.nJ + s.hop[3 * m + (c >> 1) / T];
    });

  // ---- influence matrix on u = v - ((1-c)/c) u_j:
  //      g = (u+(1), u-(1), u_z(1), div u(1)),  a = -A^{-1} g.
  //      A warp issues one FP64 instruction per ~64 cycles on GB300 whatever
  //      its active lanes, so the work is spread: step 1, one thread per
  //      (mode, tap) of the wall divergence stencil and per (mode, field) of
  //      u(1); step 2, one thread per (mode, row of A^{-1}, re/im part), the
  //      tap sum reduced over the mode's 8 lanes.  (P is free by now.)
  {
    double2* Dt = P;          // [T][9] w_q (u+ + u-)(N-9+q)
    double2* Gw = P + 9 * T;  // [T][3] u+-, u_z at the wall
    auto uv = [&](int ff, int i, int mj) {  // rows N-9.. of u+-, row N-1 of u_z
      const int c = (ff * T + mj) << 1;
      const double2 w = stage     ? UJ[(ff * N + i) * T + mj]
                        : uw_in_s ? UW[mj * 19 + (ff < 2 ? ff * 9 + i - (N - 9) : 18)]
                                  : uj(ff, i, mj);
      return double2{X[i * NT + c] - cu * w.x, X[i * NT + c + 1] - cu * w.y};
    };
    // row r of A^{-1} for the step-2 threads, loaded while step 1 runs
    double2 Ar[4];
    if (tid < 8 * T) {
      const int mj = tid >> 3, r = (tid >> 1) & 3;
      const double2* Ag = s.ainv + ((long)m * nk + min(kk0 + mj, nk - 1)) * 16 + r * 4;
#pragma unroll
      for (int c = 0; c < 4; ++c) Ar[c] = Ag[c];
    }
    if (tid < 9 * T) {
      const int mj = tid / 9, q = tid % 9, i = N - 9 + q;
      const double2 p = uv(0, i, mj), mm = uv(1, i, mj);
      const double w = wv[(N - 1) * 9 + q];
      Dt[tid] = double2{w * (p.x + mm.x), w * (p.y + mm.y)};
    } else if (tid < 12 * T) {
      const int e = tid - 9 * T, mj = e / 3, f = e % 3;
      Gw[e] = uv(f, N - 1, mj);
    }
    __syncthreads();
    if (tid < 8 * T) {  // whole warps (T >= 4)
      const int mj = tid >> 3, l = tid & 7, r = (tid >> 1) & 3, part = tid & 1;
      double2 sum = Dt[mj * 9 + l];
      if (l == 0) {
        const double2 t8 = Dt[mj * 9 + 8];
        sum = double2{sum.x + t8.x, sum.y + t8.y};
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o, 8);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o, 8);
      }
      const double2 g0 = Gw[mj * 3], g1 = Gw[mj * 3 + 1], g2 = Gw[mj * 3 + 2];
      const double akj = d.alpha * (min(kk0 + mj, nk - 1) - (K - 1));
      const double rp = RIp[N - 1], rm = RIm[N - 1];
      const double2 g[4] = {g0, g1, g2,
                            double2{fma(0.5, sum.x, fma(rp, g0.x, fma(rm, g1.x, -akj * g2.y))),
                                    fma(0.5, sum.y, fma(rp, g0.y, fma(rm, g1.y, akj * g2.x)))}};
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double2 A = Ar[c];
        acc = part ? fma(A.x, g[c].y, fma(A.y, g[c].x, acc)) : fma(A.x, g[c].x, fma(-A.y, g[c].y, acc));
      }
      ((double*)coef)[(mj * 4 + r) * 2 + part] = -acc;
    }
    __syncthreads();
  }

  // final value of chain c at row i: v - ((1-c)/c) u_j + basis responses
  auto final_value = [&](int i, int c) {
    const int part = c & 1, mi = (c >> 1) % T, f = (c >> 1) / T;
    const int kk = min(kk0 + mi, nk - 1), k = kk - (K - 1);
    const double* Bv = s.basis + (long)(abs(k) * M + m) * 6 * N;
    const double2 a0 = coef[mi * 4 + 0], ax = coef[mi * 4 + 1 + f];
    // u_z responses carry i sign(k): coefficient sign(k) (a0.x, -a0.y) swapped
    const double az = part ? a0.x : -a0.y;
    const double c0 = f == 2 ? (k > 0 ? az : (k < 0 ? -az : 0.0)) : (part ? a0.y : a0.x);
    const double c1 = part ? ax.y : ax.x;
    const double2 w = stage ? UJ[(f * N + i) * T + mi] : a.Uj[f * fs + base + (long)i * nk + kk];
    const double* B = stage ? BS + (long)mi * 6 * N : Bv;
    return X[i * NT + c] - cu * (part ? w.y : w.x) + c0 * B[i * 6 + f] + c1 * B[i * 6 + 3 + f];
  };

  // ---- fixed flux on (0,0): beta' so that 2 pi int u_z r dr = pi/2
  const bool has_mean = (m == 0 && kk0 <= K - 1 && K - 1 < kk0 + T);
  const int cz = (2 * T + (K - 1 - kk0)) << 1;  // chain (u_z, mode k=0, re)
  if (has_mean) {
    if (tid < 32) {  // warp 0 (full: NB >= 96)
      double q = 0.0;
      for (int i = tid; i < N; i += 32) q += s.wq[i] * final_value(i, cz);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if (tid == 0) {
        const double bp = (0.25 - q) / s.prm[kPrmSumWG];
        misc[0] = bp;
        *a.beta_p = bp;
      }
    }
    __syncthreads();
  }
  const double bp = has_mean ? misc[0] : 0.0;

  grid_dep_trigger_at(d, 2);
  // ---- write out (coalesced over k)
#pragma unroll 4
  for (int e = tid; e < N * NT; e += NB) {
    const int c = e % NT, i = e / NT;
    const int part = c & 1, mi = (c >> 1) % T, f = (c >> 1) / T;
    if (kk0 + mi >= nk) continue;
    double v = final_value(i, c);
    if (has_mean && c == cz) v += bp * s.G[i];
    double* out = (double*)(a.Uout + f * fs + base + (long)i * nk + kk0 + mi) + part;
    *out = v;
    if (a.curl) X[i * NT + c] = v;  // (only this element's own X is read above)
  }

  // ---- the curl of the new state (A1) for the next nonlinear evaluation, from
  //      the block's radial columns (S and P are free: u_r, u_theta; the FP32
  //      u_theta of the mixed-precision curl sits in the tail of shared memory).
  //      The mixed-precision form (curl 2) is built into the 4-mode tile only:
  //      the library's steps take it from k_curl, and in the larger tiles its
  //      code made the solve spill more registers.
  constexpr bool kMixedCurl = T == 4;
  if (a.curl) {
    __syncthreads();
    double2* UR = S;
    double2* UT = P;
    const int c0 = mi_t << 1, c1 = (T + mi_t) << 1, c2 = (2 * T + mi_t) << 1;
    for (int i = tid / T; i < N; i += NB / T) {
      const double* xr = X + i * NT;
      const double2 up = double2{xr[c0], xr[c0 + 1]}, um = double2{xr[c1], xr[c1 + 1]};
      const double2 ut = double2{0.5 * (up.y - um.y), -0.5 * (up.x - um.x)};
      UR[i * T + mi_t] = double2{0.5 * (up.x + um.x), 0.5 * (up.y + um.y)};
      UT[i * T + mi_t] = ut;
      if (kMixedCurl && a.curl == 2) UT32[i * T + mi_t] = float2{(float)ut.x, (float)ut.y};  // (curl 2 only)
    }
    __syncthreads();
    const int kk = kk0 + mi_t;
    if (kk < nk) {
      auto uz_at = [&](int i) { return double2{X[i * NT + c2], X[i * NT + c2 + 1]}; };
      auto ut_at = [&](int i) { return UT[i * T + mi_t]; };
      auto ut32_at = [&](int i) { return UT32[i * T + mi_t]; };
      for (int i = tid / T; i < N; i += NB / T) {
        if (kMixedCurl && a.curl == 2)
          curl_point<float2, true>(d, m, kk, i, ak_t, W1, s.d1f, s.r, RI, uz_at, ut_at, ut32_at, UR[i * T + mi_t],
                                   UT[i * T + mi_t], uz_at(i), (float2*)a.W6, a.Nlin);
        else
          curl_point<double2, false>(d, m, kk, i, ak_t, W1, s.d1f, s.r, RI, uz_at, ut_at, ut32_at,
                                     UR[i * T + mi_t], UT[i * T + mi_t], uz_at(i), (double2*)a.W6, nullptr);
      }
    }
  }
}

static size_t solve_smem(int N, int T);

// Tile of T modes: 4 keeps every warp of the sequential phases full (8
// right-hand sides per warp) with the most blocks; 8 when there are many
// modes per SM and two blocks of the tile still fit on an SM (so that one
// block's sequential phases overlap another's).  Measured on the ensemble's
// groups, 16 was never faster than 8 (N=32: 827 vs 767 us per launch); the
// autotuner and option "tile" can still choose it.
static int solve_tile(const Dims& d) {
  if (d.tile == 4 || d.tile == 8 || d.tile == 16) return d.tile;
  const long modes = (long)d.nk * d.M * d.B;
  if (modes / 8 >= 4 * 152 && solve_smem(d.N, 8) <= 110 * 1024) return 8;
  return 4;
}

size_t solve_smem_bytes(int N, int T) { return solve_smem(N, T); }

static size_t solve_smem(int N, int T) {
  return solve_stage_fits(N, T) ? solve_smem_staged(N, T) : solve_smem_base(N, T);
}

// Stage u_j and the responses when the staged block fits and the SM still
// holds as many blocks as the grid can use (so staging never costs occupancy).
static bool solve_use_stage(const Dims& d, int T, long blocks, bool sp = false) {
  if (!solve_stage_fits(d.N, T)) return false;
  struct SmInfo {
    int sms = 1, smem_sm = 0;
  };
  static const SmInfo info = [] {  // (thread-safe one-time initialisation)
    SmInfo i;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&i.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&i.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (i.sms <= 0) i.sms = 1;
    return i;
  }();
  const int sms = info.sms, smem_sm = info.smem_sm;
  const size_t reserve = 1024;  // per-block shared memory the system keeps
  const long with = (long)(smem_sm / (solve_smem_staged(d.N, T, sp) + reserve));
  const long without = (long)(smem_sm / (solve_smem_base(d.N, T, sp) + reserve));
  const long need = (blocks + sms - 1) / sms;
  return with >= std::min(need, without);
}

// Chunk sizes keep every transform block within ~96 KB of shared memory (two
// blocks per SM) and give each transform kernel at least two blocks per SM
// (smaller chunks, same arithmetic per column).
void choose_chunks(Dims* d) {
  const size_t budget = 96 * 1024, vb = sizeof(double2);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long target = 2L * sms;
  auto blocks = [&](int extent, int chunk, long rest) { return (long)((extent + chunk - 1) / chunk) * rest; };
  d->mcz = 8;
  while (d->mcz > 1 && (zsynth_smem(*d, d->mcz, vb) > budget || blocks(d->M, d->mcz, 6L * d->N * d->B) < target))
    d->mcz /= 2;
  d->mca = 8;
  while (d->mca > 1 && (zanalysis_smem(*d, d->mca, vb) > budget || blocks(d->M, d->mca, (long)d->N * d->B) < target))
    d->mca /= 2;
  d->zc = 4;
  while (d->zc > 1 && (product_smem(*d, d->zc, vb) > budget || blocks(d->nz, d->zc, (long)d->N * d->B) < target))
    d->zc /= 2;
}

// The dynamic shared-memory limit is a per-kernel, process-wide attribute, so
// it is raised to the device's opt-in maximum (never lowered): handles of
// different sizes then never restrict one another.
bool prepare_kernel_attrs(const Dims& d) {
  const size_t vb = sizeof(double2);
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const size_t lim = (size_t)optin;
  if (zsynth_smem(d, d.mcz, vb) > lim || zanalysis_smem(d, d.mca, vb) > lim || curl_smem(d) > lim ||
      product_smem(d, d.zc, vb) > lim || solve_smem(d.N, solve_tile(d)) > lim)
    return false;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  bool ok = cudaFuncSetAttribute(k_curl<double2, false>, a, optin) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_curl<float2, true>, a, optin) == cudaSuccess;
  with_fft_length(d.nz, [&](auto n) {
    constexpr int L = decltype(n)::value;
    ok = ok && cudaFuncSetAttribute(k_zsynth<double2, L>, a, optin) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_zanalysis<double2, L>, a, optin) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_zsynth<float2, L>, a, optin) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_zanalysis<float2, L>, a, optin) == cudaSuccess;
  });
  with_fft_length(d.nth, [&](auto n) {
    constexpr int L = decltype(n)::value;
    ok = ok && cudaFuncSetAttribute(k_product<double2, L>, a, optin) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_product<float2, L>, a, optin) == cudaSuccess;
  });
  ok = ok && cudaFuncSetAttribute(k_solve<16>, a, optin) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_solve<8>, a, optin) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_solve<4>, a, optin) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_solve<4, true>, a, optin) == cudaSuccess;
  auto fusable = [](int n) { return n == 48 || n == 72 || n == 96; };
  if (fusable(d.nz) && fusable(d.nth))  // (the option or the autotuner may switch the fused launch on later)
    with_fused_lengths(d.nz, d.nth, [&](auto z, auto t) {
      ok = ok && cudaFuncSetAttribute(k_nl_fused32<decltype(z)::value, decltype(t)::value>, a, optin) == cudaSuccess;
    });
  return ok;
}

// Shared-memory limits of the FP64 nonlinear-term kernels only (curl, z
// synthesis, theta product, z analysis) for the allocation-free entry point:
// checks their footprints against the opt-in limit and raises their dynamic
// shared-memory limit to it.
bool prepare_nonlinear_attrs(const Dims& d) {
  const size_t vb = sizeof(double2);
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const size_t lim = (size_t)optin;
  if (zsynth_smem(d, d.mcz, vb) > lim || zanalysis_smem(d, d.mca, vb) > lim || curl_smem(d) > lim ||
      product_smem(d, d.zc, vb) > lim)
    return false;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  bool ok = cudaFuncSetAttribute(k_curl<double2, false>, a, optin) == cudaSuccess;
  with_fft_length(d.nz, [&](auto n) {
    constexpr int L = decltype(n)::value;
    ok = ok && cudaFuncSetAttribute(k_zsynth<double2, L>, a, optin) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_zanalysis<double2, L>, a, optin) == cudaSuccess;
  });
  with_fft_length(d.nth, [&](auto n) {
    constexpr int L = decltype(n)::value;
    ok = ok && cudaFuncSetAttribute(k_product<double2, L>, a, optin) == cudaSuccess;
  });
  return ok;
}

void launch_solve(const Dims& d, const DevSetup& s, const SolveArgs& a, int nJ, cudaStream_t st) {
  const int T = solve_tile(d);
  const bool sp = d.spike && T == 4 && s.luH2;  // the split solve (one-wave grids, factors built)
  dim3 g((d.nk + T - 1) / T, d.M, d.B);
  const bool stage = solve_use_stage(d, T, (long)g.x * g.y * g.z, sp);
  SolveDev sd{s.d1,  s.rinv, s.wq,   s.hop,  s.luH,  s.luP,  s.basis, s.ainv, s.G,  s.prm,
              nJ,    stage ? 1 : 0,  s.d1f,  s.r,    s.luH2, s.luP2, s.spkH,  s.spkP, s.rH, s.rP};
  const size_t sm = (stage ? solve_smem_staged(d.N, T, sp) : solve_smem_base(d.N, T, sp)) +
                    (a.curl == 2 ? solve_smem_curl32(d.N, T) : 0);
  if (T == 16) launch_step_kernel(d, k_solve<16>, g, dim3(24 * 16), sm, st, d, sd, a);
  else if (T == 8) launch_step_kernel(d, k_solve<8>, g, dim3(24 * 8), sm, st, d, sd, a);
  else if (sp) launch_step_kernel(d, k_solve<4, true>, g, dim3(48 * 4), sm, st, d, sd, a);
  else launch_step_kernel(d, k_solve<4>, g, dim3(24 * 4), sm, st, d, sd, a);
}

// ------------------------------------------------------------------ diagnostics
// E/E_lam = 6 sum' w |u|^2, D/D_lam = sum' w |w|^2, I/I_lam = 4 (1 + beta) int u_z00 r dr
__global__ void __launch_bounds__(256) k_energy(Dims d, const double* __restrict__ wq,
                                                const double2* __restrict__ W6, double* partial) {
  __shared__ double su[256], sw[256];
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double eu = 0.0, ew = 0.0;
  if (idx < d.F) {
    const int n = (idx / d.nk) % d.N;
    const int m = idx / ((long)d.nk * d.N);
    const double w = (m == 0 ? 1.0 : 2.0) * wq[n];
    for (int f = 0; f < 3; ++f) {
      const double2 u = W6[f * d.F + idx], o = W6[(3 + f) * d.F + idx];
      eu += u.x * u.x + u.y * u.y;
      ew += o.x * o.x + o.y * o.y;
    }
    eu *= w;
    ew *= w;
  }
  su[threadIdx.x] = eu;
  sw[threadIdx.x] = ew;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      su[threadIdx.x] += su[threadIdx.x + h];
      sw[threadIdx.x] += sw[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = su[0];
    partial[2 * blockIdx.x + 1] = sw[0];
  }
}

__global__ void k_energy_final(Dims d, const double* __restrict__ partial, int nblk,
                               const double* __restrict__ wq, const double2* __restrict__ U,
                               const double* beta_p, const double* prm, double* out3) {
  __shared__ double su[256], sw[256], sq[256];
  double a = 0.0, b = 0.0, q = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  const double2* uz = U + 2 * d.F + (d.K - 1);  // (k,m) = (0,0), u_z: the flux int u_z r dr
  for (int n = threadIdx.x; n < d.N; n += blockDim.x) q += wq[n] * uz[(long)n * d.nk].x;
  su[threadIdx.x] = a;
  sw[threadIdx.x] = b;
  sq[threadIdx.x] = q;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      su[threadIdx.x] += su[threadIdx.x + h];
      sw[threadIdx.x] += sw[threadIdx.x + h];
      sq[threadIdx.x] += sq[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double beta = *beta_p * prm[kPrmRe] / 4.0;
    out3[0] = 6.0 * su[0];
    out3[1] = 4.0 * (1.0 + beta) * sq[0];
    out3[2] = sw[0];
  }
}

int energy_blocks(const Dims& d) { return (int)((d.F + 255) / 256); }

void launch_energy(const Dims& d, const DevSetup& s, const double2* U, const double2* W6,
                   const double* beta_p, double* partial, int nblk, double* out3, cudaStream_t st) {
  k_energy<<<nblk, 256, 0, st>>>(d, s.wq, W6, partial);
  k_energy_final<<<1, 256, 0, st>>>(d, partial, nblk, s.wq, U, beta_p, s.prm, out3);
}

// Boundary vector g of section 2 over all modes: max |u(1)| and max |div u(1)|.
__global__ void k_wall(Dims d, const double* __restrict__ d1, const double2* __restrict__ U,
                       unsigned long long* out2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.M * d.nk) return;
  const int m = idx / d.nk, kk = idx % d.nk, N = d.N;
  const long fs = d.F;
  const double2* up = U + ((long)m * N) * d.nk + kk;
  const double2* um = up + fs;
  const double2* uz = up + 2 * fs;
  const long w = (long)(N - 1) * d.nk;
  const double2 a = up[w], b = um[w], c = uz[w];
  const double ur = hypot(0.5 * (a.x + b.x), 0.5 * (a.y + b.y));
  const double ut = hypot(0.5 * (a.y - b.y), 0.5 * (a.x - b.x));
  const double umax = fmax(fmax(ur, ut), hypot(c.x, c.y));
  atomicMax(out2, __double_as_longlong(umax));
  if (m == 0 && kk == d.K - 1) return;
  const int mt = d.m_p * m;
  const double ak = d.alpha * (kk - (d.K - 1));
  const double* wr = d1 + ((long)((mt & 1) ^ 1) * N + N - 1) * 9;
  double sx = 0.0, sy = 0.0;
  for (int q = 0; q < 9; ++q) {
    const long o = (long)(N - 9 + q) * d.nk;
    sx += wr[q] * (up[o].x + um[o].x);
    sy += wr[q] * (up[o].y + um[o].y);
  }
  const double dx = 0.5 * sx + 0.5 * ((1 + mt) * a.x + (1 - mt) * b.x) - ak * c.y;
  const double dy = 0.5 * sy + 0.5 * ((1 + mt) * a.y + (1 - mt) * b.y) + ak * c.x;
  atomicMax(out2 + 1, __double_as_longlong(hypot(dx, dy)));
}

void launch_wall(const Dims& d, const DevSetup& s, const double2* U, double* out2, cudaStream_t st) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  const int nm = d.M * d.nk;
  k_wall<<<(nm + 127) / 128, 128, 0, st>>>(d, s.d1, U, (unsigned long long*)out2);
}

__global__ void k_nan(const double* __restrict__ x, long n, int* flag) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) {
      atomicOr(flag, 1);
      return;
    }
}

void launch_nan_check(const double* x, long n, int* flag, cudaStream_t st) {
  cudaMemsetAsync(flag, 0, sizeof(int), st);
  k_nan<<<304, 256, 0, st>>>(x, n, flag);
}

}  // namespace opf
