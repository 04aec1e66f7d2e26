// Batched mixed-radix FFTs in shared memory (Stockham autosort, radices
// 2, 3, 4, 5), used for the Eq. 1 transforms on the 3K x 3M grid.
//
// A block transforms `batch` sequences of length p.n stored at stride `ld`
// (complex elements) in buffer a, ping-ponging with buffer b; the returned
// pointer is whichever buffer holds the result.  sign = +1 synthesises
// (sum_k X_k e^{+2 pi i jk/n}), sign = -1 analyses; no scaling.
// tw[t] = e^{+2 pi i t/n}, t < n, in shared or global memory.
#pragma once
#include <cuda_runtime.h>

#include "opf_internal.h"

namespace opf {

template <typename V> struct Scalar;
template <> struct Scalar<double2> { using T = double; };
template <> struct Scalar<float2> { using T = float; };

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by s*i (s = +-1)
template <typename V>
__device__ __forceinline__ V cmul_si(V a, int s) { return s > 0 ? V{-a.y, a.x} : V{a.y, -a.x}; }
template <typename V, typename T>
__device__ __forceinline__ V cscale(V a, T f) { return V{a.x * f, a.y * f}; }

// In-place DFT of size R on v[0..R-1] with kernel e^{sign 2 pi i tq/R}.
template <int R, typename V>
__device__ __forceinline__ void butterfly(V* v, int sign) {
  using T = typename Scalar<V>::T;
  if constexpr (R == 2) {
    const V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const V c = cadd(v[1], v[3]), d = cmul_si(csub(v[1], v[3]), sign);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  } else if constexpr (R == 3) {
    const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
    const V t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    const V base = V{v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y};
    const V rot = cmul_si(cscale(t2, h), sign);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(base, rot);
    v[2] = csub(base, rot);
  } else if constexpr (R == 5) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    const V t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const V t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    const V a1 = V{v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
    const V a2 = V{v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
    const V b1 = cmul_si(V{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y}, sign);
    const V b2 = cmul_si(V{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y}, sign);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
}

template <int R, typename V>
__device__ __forceinline__ void fft_stage(const V* __restrict__ a, V* __restrict__ b, int n, int ld,
                                          int batch, int Ns, const V* __restrict__ tw, int sign) {
  const int nR = n / R;
  const int work = batch * nR;
  const int step = n / (Ns * R);
  for (int w = threadIdx.x; w < work; w += blockDim.x) {
    const int bt = w / nR;
    const int j = w - bt * nR;
    const int jm = j % Ns;
    const V* src = a + bt * ld;
    V* dst = b + bt * ld;
    V v[R];
    v[0] = src[j];
#pragma unroll
    for (int q = 1; q < R; ++q) {
      V t = tw[q * jm * step];
      if (sign < 0) t.y = -t.y;
      v[q] = cmul(src[j + q * nR], t);
    }
    butterfly<R>(v, sign);
    const int d0 = (j / Ns) * Ns * R + jm;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[d0 + q * Ns] = v[q];
  }
}

template <typename V>
__device__ V* block_fft(V* a, V* b, int batch, int ld, const FftPlan& p, const V* tw, int sign) {
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.rad[s];
    switch (R) {
      case 2: fft_stage<2>(a, b, p.n, ld, batch, Ns, tw, sign); break;
      case 3: fft_stage<3>(a, b, p.n, ld, batch, Ns, tw, sign); break;
      case 4: fft_stage<4>(a, b, p.n, ld, batch, Ns, tw, sign); break;
      default: fft_stage<5>(a, b, p.n, ld, batch, Ns, tw, sign); break;
    }
    __syncthreads();
    V* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

}  // namespace opf
