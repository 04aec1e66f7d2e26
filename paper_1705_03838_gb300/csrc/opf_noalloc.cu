// opf_nonlinear_noalloc: the nonlinear-term evaluation of opf_nonlinear with
// every intermediate placed in one file-scope device array instead of
// memory from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory at the point of
// the call -- a serving process whose device memory is entirely handed out
// by its own pool, code that may not trigger the device-wide synchronisation
// cudaMalloc/cudaFree can cause, or a loop that forbids allocation after
// start-up.  They pass device input and output buffers; everything else
// lives in g_noalloc_scratch below.
//
// Limits and sharing:
//  * g_noalloc_scratch holds kNoallocScratchBytes (16 MiB) on every GPU that
//    loads the library, for the life of the process.  Sizes whose working set
//    does not fit are rejected with OPF_EINVAL before any launch.
//  * All calls share the array and it keeps the last call's contents.  Every
//    region is fully written before it is read within a call, so nothing has
//    to start at zero.  Calls whose GPU work overlaps (different streams or
//    threads without ordering) race on the array.
//  * The first call on a device looks up the array's device address there
//    (cudaGetSymbolAddress) and sets the kernels' shared-memory limits; make
//    that first call before any stream capture.  CUDA loads modules lazily,
//    so it is also that first call (not loading the library) that places the
//    16 MiB array and the kernels' code on the device: make it at start-up,
//    before the caller's own pool takes the device memory.
//  * The call waits for its result (it synchronises the stream) before it
//    returns, so it refuses, with OPF_EINVAL and before launching anything,
//    a stream that is being captured.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "opf_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = 16u << 20;
constexpr int kMaxDevices = 64;

// Scratch for the no-allocation entry point.  In host code this name is only
// a stand-in for the symbol; kernels get the device address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

void* g_scratch_addr[kMaxDevices] = {nullptr};

// Transform lengths (3K, 3M) whose kernels already have their shared-memory
// limit raised, per device, in a fixed table (no host allocation either); the
// attributes are set once per device and shape (every call, once the table
// is full).
constexpr int kAttrSlots = 32;
std::mutex g_attr_mutex;
long g_attr_done[kMaxDevices][kAttrSlots] = {};
int g_attr_count[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

bool smooth235(int n) {
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Radial points, 9-point first-derivative stencils for both axis parities
// (Fornberg's recursion, same points and folding as the handle's setup) and
// the z / theta twiddle tables, computed on the device into the scratch.
__global__ void k_noalloc_consts(int N, int nz, int nth, double Re, double* prm, double* d1,
                                 double* rinv, double2* twz, double2* twth) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < opf::kPrmCount) prm[t] = t == opf::kPrmRe ? Re : 0.0;
  if (t < nz) {
    double s, c;
    sincospi(2.0 * t / nz, &s, &c);
    twz[t] = double2{c, s};
  }
  if (t < nth) {
    double s, c;
    sincospi(2.0 * t / nth, &s, &c);
    twth[t] = double2{c, s};
  }
  if (t >= N) return;
  auto rad = [&](int j) { return j == N - 1 ? 1.0 : cospi((double)(N - 1 - j) / (2.0 * N - 1.0)); };
  rinv[t] = 1.0 / rad(t);
  const int q = N + t;
  const int e0 = (q + 4 > 2 * N - 1) ? 2 * N - 9 : q - 4;
  const int lo = min(max(t - 4, 0), N - 9);
  double x[9], c[9][3];
  for (int u = 0; u < 9; ++u) {
    const int e = e0 + u;
    x[u] = e < N ? -rad(N - 1 - e) : rad(e - N);
  }
  const double z = rad(t);
  for (int u = 0; u < 9; ++u) c[u][0] = c[u][1] = c[u][2] = 0.0;
  double c1 = 1.0, c4 = x[0] - z;
  c[0][0] = 1.0;
  for (int i = 1; i < 9; ++i) {
    const int mn = min(i, 2);
    double c2 = 1.0;
    const double c5 = c4;
    c4 = x[i] - z;
    for (int j = 0; j < i; ++j) {
      const double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k) c[i][k] = c1 * (k * c[i - 1][k - 1] - c5 * c[i - 1][k]) / c2;
        c[i][0] = -c1 * c5 * c[i - 1][0] / c2;
      }
      for (int k = mn; k >= 1; --k) c[j][k] = (c4 * c[j][k] - k * c[j][k - 1]) / c3;
      c[j][0] = c4 * c[j][0] / c3;
    }
    c1 = c2;
  }
  for (int par = 0; par < 2; ++par)
    for (int u = 0; u < 9; ++u) d1[(par * N + t) * 9 + u] = 0.0;
  for (int u = 0; u < 9; ++u) {
    const int e = e0 + u;
    const bool ghost = e < N;
    const int slot = (ghost ? N - 1 - e : e - N) - lo;
    d1[(0 * N + t) * 9 + slot] += c[u][1];
    d1[(1 * N + t) * 9 + slot] += ghost ? -c[u][1] : c[u][1];
  }
}

int fail(int code, const std::string& m) {
  opf::set_last_error(m);  // reported by opf_last_error()
  return code;
}

}  // namespace

extern "C" int opf_nonlinear_noalloc(int N, int K, int M, int m_p, double alpha, double Re,
                                     const double* d_state, double* d_out, void* stream) {
  if (N < 9 || K < 1 || M < 1 || m_p < 1 || !(alpha > 0) || !(Re > 0))
    return fail(OPF_EINVAL, "opf_nonlinear_noalloc: need N>=9, K>=1, M>=1, m_p>=1, alpha>0, Re>0");
  if (!d_state || !d_out) return fail(OPF_EINVAL, "opf_nonlinear_noalloc: NULL buffer");
  if (!smooth235(3 * K) || !smooth235(3 * M))
    return fail(OPF_EINVAL, "opf_nonlinear_noalloc: 3K and 3M must have no prime factor other than 2, 3, 5");
  opf::Dims d{};
  d.N = N;
  d.K = K;
  d.M = M;
  d.m_p = m_p;
  d.nk = 2 * K - 1;
  d.nz = 3 * K;
  d.nth = 3 * M;
  d.inv_grid = 1.0 / ((double)d.nz * d.nth);
  d.alpha = alpha;
  d.Re = Re;
  d.dt = 1.0;
  d.c = 0.5;
  d.F = (long)M * N * d.nk;
  opf::choose_chunks(&d);
  opf::FftPlan pz{}, pth{};
  if (!opf::make_plan(d.nz, &pz) || !opf::make_plan(d.nth, &pth))
    return fail(OPF_EINVAL, "opf_nonlinear_noalloc: no FFT plan for 3K or 3M");

  // scratch layout: constants | U (3F) | W6 (6F) | Z6 (6P) | ZN (3P) | N (3F)
  const size_t F16 = (size_t)d.F * sizeof(double2);
  const size_t P16 = (size_t)N * d.nz * M * sizeof(double2);
  const size_t o_prm = 0;
  const size_t o_d1 = align256(o_prm + opf::kPrmCount * sizeof(double));
  const size_t o_rinv = align256(o_d1 + 2 * (size_t)N * 9 * sizeof(double));
  const size_t o_twz = align256(o_rinv + N * sizeof(double));
  const size_t o_twth = align256(o_twz + d.nz * sizeof(double2));
  const size_t o_U = align256(o_twth + d.nth * sizeof(double2));
  const size_t o_W6 = align256(o_U + 3 * F16);
  const size_t o_Z6 = align256(o_W6 + 6 * F16);
  const size_t o_ZN = align256(o_Z6 + 6 * P16);
  const size_t o_N = align256(o_ZN + 3 * P16);
  const size_t need = align256(o_N + 3 * F16);
  if (need > kNoallocScratchBytes)
    return fail(OPF_EINVAL, "opf_nonlinear_noalloc: resolution needs " + std::to_string(need) +
                                " bytes of scratch, more than the fixed " +
                                std::to_string(kNoallocScratchBytes));

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(OPF_ECUDA, "opf_nonlinear_noalloc: no usable CUDA device");
  cudaStream_t st = (cudaStream_t)stream;
  {  // the call ends with a stream synchronisation, which a capture forbids
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
      if (e != cudaSuccess) cudaGetLastError();  // leave no sticky status behind
      return fail(OPF_EINVAL, "opf_nonlinear_noalloc: the stream is being captured (or its capture state "
                              "cannot be read); this call synchronises its stream and cannot run inside a capture");
    }
  }
  if (!g_scratch_addr[dev]) {  // once per device, with that device current
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(OPF_ECUDA, std::string("opf_nonlinear_noalloc: cudaGetSymbolAddress: ") +
                                 cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  {
    const long key = (long)d.nz << 20 | d.nth;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    long* done = g_attr_done[dev];
    int& count = g_attr_count[dev];
    if (std::find(done, done + count, key) == done + count) {
      if (!opf::prepare_nonlinear_attrs(d))
        return fail(OPF_EINVAL, "opf_nonlinear_noalloc: resolution needs more shared memory than a block has");
      if (count < kAttrSlots) done[count++] = key;
    }
  }
  unsigned char* base = (unsigned char*)g_scratch_addr[dev];
  opf::DevSetup s{};
  s.prm = (double*)(base + o_prm);
  d.prm = s.prm;
  s.d1 = (double*)(base + o_d1);
  s.rinv = (double*)(base + o_rinv);
  s.tw_z = (double2*)(base + o_twz);
  s.tw_th = (double2*)(base + o_twth);
  double2* U = (double2*)(base + o_U);
  double2* W6 = (double2*)(base + o_W6);
  double2* Z6 = (double2*)(base + o_Z6);
  double2* ZN = (double2*)(base + o_ZN);
  double2* Nn = (double2*)(base + o_N);

  const int nc = std::max(N, std::max(d.nz, d.nth));
  k_noalloc_consts<<<(nc + 127) / 128, 128, 0, st>>>(N, d.nz, d.nth, Re, s.prm, s.d1, s.rinv, s.tw_z,
                                                      s.tw_th);
  opf::launch_abi_to_internal(d, (const double2*)d_state, U, st);
  opf::launch_curl(d, s, U, W6, st);
  opf::launch_zsynth(d, s, pz, W6, Z6, st);
  opf::launch_product(d, s, pth, Z6, ZN, st);
  opf::launch_zanalysis(d, s, pz, ZN, Nn, st);
  opf::launch_internal_to_abi(d, Nn, (double2*)d_out, 1, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fail(OPF_ECUDA, std::string("opf_nonlinear_noalloc: ") + cudaGetErrorString(e));
  return OPF_OK;
}
