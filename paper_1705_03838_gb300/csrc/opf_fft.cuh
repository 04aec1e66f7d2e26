// Batched mixed-radix FFTs in shared memory (Stockham autosort, radices
// 2, 3, 4, 5, 8), used for the Eq. 1 transforms on the 3K x 3M grid.
//
// A block transforms `batch` sequences of length p.n stored at stride `ld`
// (complex elements) in buffer a, ping-ponging with buffer b; the returned
// pointer is whichever buffer holds the result.  sign = +1 synthesises
// (sum_k X_k e^{+2 pi i jk/n}), sign = -1 analyses; no scaling.
// tw[t] = e^{+2 pi i t/n}, t < n, in shared or global memory.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

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
// Radix 8 with v[3] = v[4] = 0 (the first stage of a synthesis whose middle
// third is the zero padding of the 3/2 rule): the same outputs as
// butterfly<8> without the additions of the two zero inputs.
template <typename V>
__device__ __forceinline__ void butterfly8_zm(V* v, int sign) {
  using T = typename Scalar<V>::T;
  // even points (v0, v2, 0, v6)
  const V ec = cadd(v[2], v[6]), ed = cmul_si(csub(v[2], v[6]), sign);
  V e[4] = {cadd(v[0], ec), cadd(v[0], ed), csub(v[0], ec), csub(v[0], ed)};
  // odd points (v1, 0, v5, v7)
  const V oa = cadd(v[1], v[5]), ob = csub(v[1], v[5]);
  const V od = cmul_si(V{-v[7].x, -v[7].y}, sign);
  V o[4] = {cadd(oa, v[7]), cadd(ob, od), csub(oa, v[7]), csub(ob, od)};
  const T h = (T)0.70710678118654752440;  // 1 / sqrt(2)
  const T s = (T)sign;
  const V o1 = V{h * (o[1].x - s * o[1].y), h * (o[1].y + s * o[1].x)};
  const V o2 = cmul_si(o[2], sign);
  const V o3 = V{-h * (o[3].x + s * o[3].y), h * (s * o[3].x - o[3].y)};
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

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
  } else if constexpr (R == 8) {
    // two radix-4 transforms of the even and odd points, joined by the
    // eighth roots of unity w^q = e^{sign 2 pi i q/8}
    V e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    butterfly<4>(e, sign);
    butterfly<4>(o, sign);
    const T h = (T)0.70710678118654752440;  // 1 / sqrt(2)
    const T s = (T)sign;
    const V o1 = V{h * (o[1].x - s * o[1].y), h * (o[1].y + s * o[1].x)};
    const V o2 = cmul_si(o[2], sign);
    const V o3 = V{-h * (o[3].x + s * o[3].y), h * (s * o[3].x - o[3].y)};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
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

// ---------------------------------------------------------------------------
// The same Stockham transform for a length N known at compile time (the
// common grid lengths 3K, 3M): radices, strides and the twiddle stride are
// constants, so the index arithmetic folds into shifts and multiply-highs, the
// first stage (all twiddles 1) skips its multiplications, and radix 8 cuts the
// number of shared-memory passes.  Same conventions as block_fft.
//
// The buffers between two stages hold element i of a sequence at
// fft_swz(i) = i ^ ((i >> 3) & 7) (a permutation inside each group of eight;
// every compiled length is a multiple of 8): the first stage writes element
// j R + q for consecutive j, a stride of R complex values that would put a
// warp's stores on two or four of the 16 eight-byte bank pairs, and the
// permutation spreads them.  The caller's input and the result are in the
// plain layout; the arithmetic is unchanged.
__host__ __device__ constexpr int fft_swz(int i) { return i ^ ((i >> 3) & 7); }

template <int R, int N, int NS, int SIGN, bool SWR, bool SWW, bool ZM, typename V>
__device__ __forceinline__ void fft_stage_c(const V* __restrict__ a, V* __restrict__ b, int ld, int batch,
                                            const V* __restrict__ tw) {
  constexpr bool zm = ZM && NS == 1 && R == 8;  // inputs 3 and 4 lie in the zero middle third
  static_assert(N % 8 == 0, "the swizzle permutes groups of eight");
  constexpr int nR = N / R, step = N / (NS * R);
  const int work = batch * nR;
  for (int w = threadIdx.x; w < work; w += blockDim.x) {
    const int bt = w / nR;
    const int j = w - bt * nR;
    const int jm = j % NS;
    const V* src = a + bt * ld;
    V* dst = b + bt * ld;
    V v[R];
    v[0] = src[SWR ? fft_swz(j) : j];
#pragma unroll
    for (int q = 1; q < R; ++q) {
      const int ix = j + q * nR;
      if constexpr (zm) {
        if (q == 3 || q == 4) continue;
      }
      if constexpr (NS == 1) {
        v[q] = src[SWR ? fft_swz(ix) : ix];
      } else {
        V t = tw[q * jm * step];
        if constexpr (SIGN < 0) t.y = -t.y;
        v[q] = cmul(src[SWR ? fft_swz(ix) : ix], t);
      }
    }
    if constexpr (zm) {
      butterfly8_zm(v, SIGN);
    } else {
      butterfly<R>(v, SIGN);
    }
    const int d0 = (j / NS) * NS * R + jm;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int ox = d0 + q * NS;
      dst[SWW ? fft_swz(ox) : ox] = v[q];
    }
  }
}

template <int N, int NS, int SIGN, bool ZM, int R, int... Rest, typename V>
__device__ __forceinline__ V* fft_stages_c(V* a, V* b, int ld, int batch, const V* tw) {
  constexpr bool last = sizeof...(Rest) == 0;
  fft_stage_c<R, N, NS, SIGN, (NS > 1), !last, ZM>(a, b, ld, batch, tw);
  __syncthreads();
  if constexpr (last) {
    return b;
  } else {
    return fft_stages_c<N, NS * R, SIGN, ZM, Rest...>(b, a, ld, batch, tw);
  }
}

// Element e < count of a block-wide copy: v = load(e), then store(e, v), with
// U loads in flight per thread (thread t takes e = t, t + blockDim.x, ...,
// as a plain strided loop would, so coalescing is the same).
template <int U, typename V, typename Load, typename Store>
__device__ __forceinline__ void block_copy_batched(int count, Load load, Store store) {
  for (int b = threadIdx.x; b < count; b += U * blockDim.x) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = b + u * blockDim.x;
      if (e < count) v[u] = load(e);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = b + u * blockDim.x;
      if (e < count) store(e, v[u]);
    }
  }
}

// Lengths with a compiled plan (others use block_fft).
__host__ __device__ constexpr bool fft_length_compiled(int n) {
  return n == 48 || n == 72 || n == 96 || n == 192 || n == 384;
}

// ZERO_MID: the inputs in the middle third, positions (N/3, 2N/3), are zero
// (a synthesis of the 3/2 rule); the radix-8 first stages then skip them.
template <int N, int SIGN, bool ZERO_MID = false, typename V>
__device__ __forceinline__ V* block_fft_c(V* a, V* b, int batch, int ld, const V* tw) {
  static_assert(fft_length_compiled(N), "no compiled plan for this length");
  if constexpr (N == 48) return fft_stages_c<48, 1, SIGN, ZERO_MID, 4, 4, 3>(a, b, ld, batch, tw);
  else if constexpr (N == 72) return fft_stages_c<72, 1, SIGN, ZERO_MID, 8, 3, 3>(a, b, ld, batch, tw);
  else if constexpr (N == 96) return fft_stages_c<96, 1, SIGN, ZERO_MID, 8, 4, 3>(a, b, ld, batch, tw);
  else if constexpr (N == 192) return fft_stages_c<192, 1, SIGN, ZERO_MID, 8, 8, 3>(a, b, ld, batch, tw);
  else return fft_stages_c<384, 1, SIGN, ZERO_MID, 8, 4, 4, 3>(a, b, ld, batch, tw);
}

// Calls f(std::integral_constant<int, n>) for a compiled length n, else
// f(std::integral_constant<int, 0>) (runtime plan).
template <class F>
inline void with_fft_length(int n, F&& f) {
  switch (n) {
    case 48: f(std::integral_constant<int, 48>{}); break;
    case 72: f(std::integral_constant<int, 72>{}); break;
    case 96: f(std::integral_constant<int, 96>{}); break;
    case 192: f(std::integral_constant<int, 192>{}); break;
    case 384: f(std::integral_constant<int, 384>{}); break;
    default: f(std::integral_constant<int, 0>{}); break;
  }
}

}  // namespace opf
