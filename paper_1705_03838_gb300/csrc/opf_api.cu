// C ABI of libopf (declared in include/opf.h): handle life cycle, state
// transfer, and the predictor-corrector orchestration of section 2, for one
// trajectory (opf_t) and for batched ensembles of trajectories (opf_ens_t).
//
// A Group holds B trajectories of one shape (N, K, M, m_p, alpha) in two
// device arenas -- work buffers and setup arrays -- with fixed strides, so
// every kernel launch covers all B trajectories (grid z).  A Runner records
// one time step of a list of groups as a CUDA graph and replays it.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <thread>
#include <string>
#include <tuple>
#include <vector>

#include "opf_internal.h"

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CU(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(OPF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

}  // namespace

namespace opf {
void set_last_error(const std::string& m) { g_err = m; }
}  // namespace opf

namespace {

constexpr int kMaxSlots = 128;
const char* kNames[] = {"curl", "zsynth", "product", "zanalysis", "solve", "transforms"};
constexpr int kNumNames = 6;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

bool smooth235(int n) {
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

// ------------------------------------------------------------------ Group
struct Group {
  opf::Dims d{};
  opf::FftPlan pz{}, pth{};
  int nJ = 0;
  bool shared_setup = false;
  // FP64 steps: W6 holds the curl of U, as the last solve of a step leaves
  // it; anything else that writes U, W6 or an option clears this, and the
  // next step then starts with a curl launch
  bool w6_valid = false;
  std::vector<double> Re, dt, time;  // per trajectory
  opf::DevSetup ds;                  // trajectory 0's setup arrays
  char* parena = nullptr;
  char* sarena = nullptr;
  size_t pstride = 0, sstride = 0;
  std::vector<double> mesh;  // user radial mesh (empty: the default points)
  // trajectory 0's work buffers (trajectory b: + b * sstride bytes)
  double2 *U = nullptr, *U1 = nullptr, *Nj = nullptr, *Nq = nullptr, *W6 = nullptr;
  double2 *Z6 = nullptr, *ZN = nullptr, *abi = nullptr, *tmpU = nullptr, *Nlin = nullptr;
  float2 *W6f = nullptr, *Z6f = nullptr, *ZNf = nullptr;
  double *beta_p = nullptr, *partial = nullptr, *out3 = nullptr, *out2 = nullptr;
  double* cfl = nullptr;  // per trajectory: max |u|/spacing over the grid
  int* flag = nullptr;
  int nblk_energy = 0;
  // setup-arena offsets (same for every trajectory), for in-place rebuilds
  size_t o_prm = 0, o_rinv = 0, o_d1 = 0, o_wq = 0, o_hop = 0, o_luH = 0, o_luP = 0;
  size_t o_basis = 0, o_ainv = 0, o_G = 0, o_twz = 0, o_twt = 0, o_twz32 = 0, o_twt32 = 0;
  size_t o_r = 0, o_d1f = 0;
  size_t o_luH2 = 0, o_luP2 = 0, o_spkH = 0, o_spkP = 0, o_rH = 0, o_rP = 0;
  bool spike_built = false;  // split factors built (decided once, at creation)
  bool spike_default = false;  // the split solve is on unless the option says otherwise

  template <typename P>
  P* at(P* p, int b) const {
    return (P*)((char*)p + (size_t)b * sstride);
  }
  opf::DevSetup setup_of(int b) const {
    if (shared_setup || b == 0) return ds;
    opf::DevSetup s = ds;
    const size_t o = (size_t)b * pstride;
    auto sh = [&](auto* p) { return (decltype(p))((char*)p + o); };
    s.prm = sh(s.prm);
    s.rinv = sh(s.rinv);
    s.d1 = sh(s.d1);
    s.wq = sh(s.wq);
    s.hop = sh(s.hop);
    s.luH = sh(s.luH);
    s.luP = sh(s.luP);
    s.basis = sh(s.basis);
    s.ainv = sh(s.ainv);
    s.G = sh(s.G);
    s.tw_z = sh(s.tw_z);
    s.tw_th = sh(s.tw_th);
    s.tw_z32 = sh(s.tw_z32);
    s.tw_th32 = sh(s.tw_th32);
    s.r = sh(s.r);
    s.d1f = sh(s.d1f);
    if (spike_built) {
      s.luH2 = sh(s.luH2);
      s.luP2 = sh(s.luP2);
      s.spkH = sh(s.spkH);
      s.spkP = sh(s.spkP);
      s.rH = sh(s.rH);
      s.rP = sh(s.rP);
    }
    return s;
  }
  // launch dimensions of trajectory b alone (pointers offset on the host)
  opf::Dims single(int b) const {
    opf::Dims e = d;
    e.B = 1;
    e.ss = 0;
    e.ps = 0;
    e.prm = setup_of(b).prm;
    return e;
  }
};

void group_free(Group* g) {
  if (g->sarena) cudaFree(g->sarena);
  if (g->parena) cudaFree(g->parena);
  g->sarena = g->parena = nullptr;
}

struct Layout {
  size_t off = 0;
  size_t add(size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  }
};

// Build the host setups (radial operators, LU factors, influence data) of
// every trajectory for its current Re and dt and upload them into the setup
// arena; first = true also lays the arena out and allocates it.  Rebuilding
// keeps every device address, so captured graphs stay valid.
int group_fill_setups(Group* g, bool first) {
  opf::Dims& d = g->d;
  const int N = d.N, K = d.K, M = d.M, m_p = d.m_p, B = d.B;
  const double alpha = d.alpha;
  const double* Re = g->Re.data();
  const double* dt = g->dt.data();
  const int nsetup = g->shared_setup ? 1 : B;
  // host setups, built on all host cores when trajectories differ
  std::vector<opf::Setup> hs(nsetup);
  std::vector<std::string> errs(nsetup);
  std::vector<char> ok(nsetup, 0);
  auto build_one = [&](int b) {
    opf::Setup& s = hs[b];
    s.N = N;
    s.K = K;
    s.M = M;
    s.m_p = m_p;
    s.alpha = alpha;
    s.Re = Re[b];
    s.dt = dt[b];
    s.c = 0.5;
    s.r_user = g->mesh;
    s.spike = g->spike_built;
    ok[b] = opf::build_setup(&s, &errs[b]) ? 1 : 0;
  };
  const int nthreads = std::max(1, std::min<int>(nsetup, (int)std::thread::hardware_concurrency()));
  if (nthreads == 1) {
    for (int b = 0; b < nsetup; ++b) build_one(b);
  } else {
    std::vector<std::thread> pool;
    std::atomic<int> next{0};
    for (int t = 0; t < nthreads; ++t)
      pool.emplace_back([&] {
        for (int b = next++; b < nsetup; b = next++) build_one(b);
      });
    for (auto& th : pool) th.join();
  }
  for (int b = 0; b < nsetup; ++b)
    if (!ok[b]) return fail(OPF_EINVAL, errs[b]);
  g->nJ = hs[0].nJ;

  // setup arena layout (identical sizes for every trajectory of the shape)
  const opf::Setup& s0 = hs[0];
  Layout pl;
  g->o_prm = pl.add(opf::kPrmCount * sizeof(double));
  g->o_rinv = pl.add(s0.rinv.size() * 8);
  g->o_d1 = pl.add(s0.d1.size() * 8);
  g->o_wq = pl.add(s0.wq.size() * 8);
  g->o_hop = pl.add(s0.hop.size() * sizeof(int));
  g->o_luH = pl.add(s0.luH.size() * 8);
  g->o_luP = pl.add(s0.luP.size() * 8);
  g->o_basis = pl.add(s0.basis.size() * 8);
  g->o_ainv = pl.add(s0.ainv.size() * 8);
  g->o_G = pl.add(s0.G.size() * 8);
  g->o_twz = pl.add(d.nz * sizeof(double2));
  g->o_twt = pl.add(d.nth * sizeof(double2));
  g->o_twz32 = pl.add(d.nz * sizeof(float2));
  g->o_twt32 = pl.add(d.nth * sizeof(float2));
  g->o_r = pl.add(s0.r.size() * 8);
  g->o_d1f = pl.add((s0.d1.size() + s0.rinv.size()) * sizeof(float));
  g->o_luH2 = pl.add(s0.luH2.size() * 8);
  g->o_luP2 = pl.add(s0.luP2.size() * 8);
  g->o_spkH = pl.add(s0.spkH.size() * 8);
  g->o_spkP = pl.add(s0.spkP.size() * 8);
  g->o_rH = pl.add(s0.rH.size() * 8);
  g->o_rP = pl.add(s0.rP.size() * 8);
  if (first) {
    g->pstride = pl.off;
    if (cudaMalloc((void**)&g->parena, g->pstride * nsetup) != cudaSuccess)
      return fail(OPF_ENOMEM, "cudaMalloc of setup arrays failed");
  }
  std::vector<char> host(g->pstride, 0);
  auto put = [&](size_t o, const void* src, size_t bytes) { std::memcpy(host.data() + o, src, bytes); };
  std::vector<double2> twz(d.nz), twt(d.nth);
  std::vector<float2> twz32(d.nz), twt32(d.nth);
  auto tw = [](int n, std::vector<double2>& t, std::vector<float2>& t32) {
    for (int i = 0; i < n; ++i) {
      const long double a = 2.0L * 3.14159265358979323846264338327950288L * i / n;
      t[i] = double2{(double)cosl(a), (double)sinl(a)};
      t32[i] = float2{(float)t[i].x, (float)t[i].y};
    }
  };
  tw(d.nz, twz, twz32);
  tw(d.nth, twt, twt32);
  for (int b = 0; b < nsetup; ++b) {
    const opf::Setup& s = hs[b];
    double prm[opf::kPrmCount] = {0};
    prm[opf::kPrmRe] = s.Re;
    prm[opf::kPrmDt] = s.dt;
    prm[opf::kPrmC] = s.c;
    prm[opf::kPrmSumWG] = s.flux_G;
    prm[opf::kPrmCi] = 1.0 / (s.c * s.dt);  // the solve's scalings, divided here once
    prm[opf::kPrmCu] = (1.0 - s.c) / s.c;
    put(g->o_prm, prm, sizeof prm);
    put(g->o_rinv, s.rinv.data(), s.rinv.size() * 8);
    put(g->o_d1, s.d1.data(), s.d1.size() * 8);
    put(g->o_wq, s.wq.data(), s.wq.size() * 8);
    put(g->o_hop, s.hop.data(), s.hop.size() * sizeof(int));
    put(g->o_luH, s.luH.data(), s.luH.size() * 8);
    put(g->o_luP, s.luP.data(), s.luP.size() * 8);
    {  // device order [K][M][N][6]: the six responses of one radial row together
      const size_t nmode = s.basis.size() / (6 * (size_t)d.N);
      std::vector<double> bt(s.basis.size());
      for (size_t q = 0; q < nmode; ++q)
        for (int v = 0; v < 6; ++v)
          for (int i = 0; i < d.N; ++i) bt[(q * d.N + i) * 6 + v] = s.basis[(q * 6 + v) * d.N + i];
      put(g->o_basis, bt.data(), bt.size() * 8);
    }
    put(g->o_ainv, s.ainv.data(), s.ainv.size() * 8);
    put(g->o_G, s.G.data(), s.G.size() * 8);
    put(g->o_twz, twz.data(), d.nz * sizeof(double2));
    put(g->o_twt, twt.data(), d.nth * sizeof(double2));
    put(g->o_twz32, twz32.data(), d.nz * sizeof(float2));
    put(g->o_twt32, twt32.data(), d.nth * sizeof(float2));
    put(g->o_r, s.r.data(), s.r.size() * 8);
    std::vector<float> d1f(s.d1.begin(), s.d1.end());  // FP32 stencils, then FP32 1/r
    d1f.insert(d1f.end(), s.rinv.begin(), s.rinv.end());
    put(g->o_d1f, d1f.data(), d1f.size() * sizeof(float));
    put(g->o_luH2, s.luH2.data(), s.luH2.size() * 8);
    put(g->o_luP2, s.luP2.data(), s.luP2.size() * 8);
    put(g->o_spkH, s.spkH.data(), s.spkH.size() * 8);
    put(g->o_spkP, s.spkP.data(), s.spkP.size() * 8);
    put(g->o_rH, s.rH.data(), s.rH.size() * 8);
    put(g->o_rP, s.rP.data(), s.rP.size() * 8);
    CU(cudaMemcpy(g->parena + (size_t)b * g->pstride, host.data(), g->pstride, cudaMemcpyHostToDevice));
  }
  return OPF_OK;
}

// Build host setups, lay out and fill both arenas for B trajectories of one
// shape with per-trajectory Re and dt (one shared setup when all are equal).
int group_build(Group* g, int N, int K, int M, int m_p, double alpha, int B, const double* Re,
                const double* dt, bool separate_setups = false) {
  if (N < 9 || K < 1 || M < 1 || m_p < 1 || !(alpha > 0) || B < 1)
    return fail(OPF_EINVAL, "need N>=9, K>=1, M>=1, m_p>=1, alpha>0");
  for (int b = 0; b < B; ++b)
    if (!(Re[b] > 0) || !(dt[b] > 0)) return fail(OPF_EINVAL, "need Re>0, dt>0");
  if (!smooth235(3 * K) || !smooth235(3 * M))
    return fail(OPF_EINVAL, "3K and 3M must have no prime factor other than 2, 3, 5");
  int ndev = 0;
  const cudaError_t de = cudaGetDeviceCount(&ndev);
  if (de != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(OPF_ECUDA, std::string("no CUDA device available (") +
                               (de != cudaSuccess ? cudaGetErrorString(de) : "0 devices") + ")");
  }
  opf::Dims& d = g->d;
  d.N = N;
  d.K = K;
  d.M = M;
  d.m_p = m_p;
  d.nk = 2 * K - 1;
  d.nz = 3 * K;
  d.nth = 3 * M;
  d.inv_grid = 1.0 / ((double)d.nz * d.nth);
  d.alpha = alpha;
  d.Re = Re[0];
  d.dt = dt[0];
  d.c = 0.5;
  d.F = (long)M * N * d.nk;
  d.B = B;
  opf::choose_chunks(&d);
  if (!opf::make_plan(d.nz, &g->pz) || !opf::make_plan(d.nth, &g->pth))
    return fail(OPF_EINVAL, "no FFT plan for 3K or 3M");
  g->Re.assign(Re, Re + B);
  g->dt.assign(dt, dt + B);
  g->time.assign(B, 0.0);
  g->shared_setup = !separate_setups;
  for (int b = 1; b < B; ++b)
    if (Re[b] != Re[0] || dt[b] != dt[0]) g->shared_setup = false;
  g->nJ = 0;
  {  // split factors are built for grids of up to three 4-mode blocks per SM;
     // the split solve is the default where there is at most one (the
     // substitution chains are then the critical path, not the FP64 pipe)
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long blocks = (long)((d.nk + 3) / 4) * M * B;
    g->spike_built = N % 2 == 0 && N >= 26 && blocks <= 3L * sms;
    g->spike_default = g->spike_built && blocks <= sms;
  }
  int rc = group_fill_setups(g, true);
  if (rc) return rc;
  char* P = g->parena;
  g->ds.prm = (double*)(P + g->o_prm);
  g->ds.rinv = (double*)(P + g->o_rinv);
  g->ds.d1 = (double*)(P + g->o_d1);
  g->ds.wq = (double*)(P + g->o_wq);
  g->ds.hop = (int*)(P + g->o_hop);
  g->ds.luH = (double*)(P + g->o_luH);
  g->ds.luP = (double*)(P + g->o_luP);
  g->ds.basis = (double*)(P + g->o_basis);
  g->ds.ainv = (double2*)(P + g->o_ainv);
  g->ds.G = (double*)(P + g->o_G);
  g->ds.tw_z = (double2*)(P + g->o_twz);
  g->ds.tw_th = (double2*)(P + g->o_twt);
  g->ds.tw_z32 = (float2*)(P + g->o_twz32);
  g->ds.tw_th32 = (float2*)(P + g->o_twt32);
  g->ds.r = (double*)(P + g->o_r);
  g->ds.d1f = (float*)(P + g->o_d1f);
  if (g->spike_built) {
    g->ds.luH2 = (double*)(P + g->o_luH2);
    g->ds.luP2 = (double*)(P + g->o_luP2);
    g->ds.spkH = (double*)(P + g->o_spkH);
    g->ds.spkP = (double*)(P + g->o_spkP);
    g->ds.rH = (double*)(P + g->o_rH);
    g->ds.rP = (double*)(P + g->o_rP);
  }
  d.spike = g->spike_default ? 1 : 0;
  d.ps = g->shared_setup ? 0 : (long)g->pstride;
  d.prm = g->ds.prm;

  // work arena: FP32 intermediates alias the FP64 ones (one precision per step)
  const size_t F16 = (size_t)d.F * sizeof(double2);
  const size_t P16 = (size_t)N * d.nz * M * sizeof(double2);
  g->nblk_energy = opf::energy_blocks(d);
  Layout sl;
  const size_t o_U = sl.add(3 * F16), o_U1 = sl.add(3 * F16), o_Nj = sl.add(3 * F16);
  const size_t o_Nq = sl.add(3 * F16), o_W6 = sl.add(6 * F16), o_Z6 = sl.add(6 * P16);
  const size_t o_ZN = sl.add(3 * P16), o_abi = sl.add(3 * F16), o_tmp = sl.add(3 * F16);
  const size_t o_Nlin = sl.add(3 * F16), o_beta = sl.add(16), o_out3 = sl.add(32);
  const size_t o_out2 = sl.add(16), o_flag = sl.add(16), o_cfl = sl.add(16);
  const size_t o_part = sl.add((size_t)2 * g->nblk_energy * sizeof(double));
  g->sstride = sl.off;
  if (cudaMalloc((void**)&g->sarena, g->sstride * B) != cudaSuccess)
    return fail(OPF_ENOMEM, "cudaMalloc of work buffers failed");
  CU(cudaMemset(g->sarena, 0, g->sstride * B));
  char* S = g->sarena;
  g->U = (double2*)(S + o_U);
  g->U1 = (double2*)(S + o_U1);
  g->Nj = (double2*)(S + o_Nj);
  g->Nq = (double2*)(S + o_Nq);
  g->W6 = (double2*)(S + o_W6);
  g->Z6 = (double2*)(S + o_Z6);
  g->ZN = (double2*)(S + o_ZN);
  g->W6f = (float2*)g->W6;
  g->Z6f = (float2*)g->Z6;
  g->ZNf = (float2*)g->ZN;
  g->abi = (double2*)(S + o_abi);
  g->tmpU = (double2*)(S + o_tmp);
  g->Nlin = (double2*)(S + o_Nlin);
  g->beta_p = (double*)(S + o_beta);
  g->out3 = (double*)(S + o_out3);
  g->out2 = (double*)(S + o_out2);
  g->flag = (int*)(S + o_flag);
  g->cfl = (double*)(S + o_cfl);
  g->partial = (double*)(S + o_part);
  d.ss = (long)g->sstride;
  if (!opf::prepare_kernel_attrs(d))
    return fail(OPF_EINVAL, "resolution needs more shared memory than a block has");
  return OPF_OK;
}

// ------------------------------------------------------------------ Runner
struct Runner {
  std::vector<Group*> groups;
  cudaStream_t own = nullptr, stream = nullptr;
  int precision = 0, n_corr = 1, use_graph = 1, timing = 0;
  int autotune = 0;  // 1: time launch shapes on the next step, keep the fastest
  double cfl_C = 0.0;   // > 0: CFL-controlled time step (single trajectory)
  double dt_max = 0.0;  // upper bound of the controlled time step
  cudaGraphExec_t gexec = nullptr;
  // groups after the first run on side streams, forked from and joined back
  // into `stream` (graph branches when captured); cur: the stream the group
  // being enqueued runs on (null: stream)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join_ev;
  cudaEvent_t fork_ev = nullptr;
  cudaStream_t cur = nullptr;
  cudaStream_t st() const { return cur ? cur : stream; }
  cudaEvent_t ev[kMaxSlots][2];
  int slot_name[kMaxSlots];
  int nslots = 0, graph_nslots = 0;
  bool events_made = false;
  double tot_ms[kNumNames] = {0};
  int tot_n[kNumNames] = {0};

  // timing 1: every kernel; timing 2: only kernel `timed_kernel` (fewer event nodes)
  int timed_kernel = 4;
  bool timed(int name) const { return timing == 1 || (timing == 2 && name == timed_kernel); }
  int open_name = -1;
  void begin(int name) {
    open_name = name;
    if (!timed(name) || nslots >= kMaxSlots) return;
    slot_name[nslots] = name;
    // external: inside stream capture this becomes an event-record node
    cudaEventRecordWithFlags(ev[nslots][0], st(), cudaEventRecordExternal);
  }
  void end() {
    if (!timed(open_name) || nslots >= kMaxSlots) return;
    cudaEventRecordWithFlags(ev[nslots][1], st(), cudaEventRecordExternal);
    ++nslots;
  }
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
};

int runner_init(Runner* r) {
  CU(cudaStreamCreateWithFlags(&r->own, cudaStreamNonBlocking));
  r->stream = r->own;
  for (int i = 0; i < kMaxSlots; ++i) {
    CU(cudaEventCreate(&r->ev[i][0]));
    CU(cudaEventCreate(&r->ev[i][1]));
  }
  r->events_made = true;
  return OPF_OK;
}

void runner_free(Runner* r) {
  r->drop_graph();
  if (r->events_made)
    for (int i = 0; i < kMaxSlots; ++i) {
      cudaEventDestroy(r->ev[i][0]);
      cudaEventDestroy(r->ev[i][1]);
    }
  r->events_made = false;
  for (cudaStream_t s : r->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : r->join_ev) cudaEventDestroy(e);
  if (r->fork_ev) cudaEventDestroy(r->fork_ev);
  r->side.clear();
  r->join_ev.clear();
  r->fork_ev = nullptr;
  if (r->own) cudaStreamDestroy(r->own);
  r->own = nullptr;
}

// The curl of U (A1) into the group's W6 (and Nlin in mixed precision);
// timed: inside the per-kernel event slots.
void enqueue_curl(Runner* r, const Group& g, const double2* U, bool timed = true) {
  if (timed) r->begin(0);
  if (r->precision == 1) opf::launch_curl_split32(g.d, g.ds, U, g.W6f, g.Nlin, r->st());
  else opf::launch_curl(g.d, g.ds, U, g.W6, r->st());
  if (timed) r->end();
}

// N(U) into Nout; with_curl false: W6 already holds the curl of U.
void enqueue_nonlinear(Runner* r, const Group& g, const double2* U, double2* Nout, bool with_curl = true) {
  const opf::Dims& d = g.d;
  cudaStream_t st = r->st();
  if (with_curl) enqueue_curl(r, g, U);
  if (r->precision == 1) {
    if (opf::fused32_cluster(d)) {  // the three transforms as one cluster launch
      r->begin(5);
      opf::launch_nl_fused32(d, g.ds, g.W6f, g.Nlin, Nout, st);
      r->end();
      return;
    }
    r->begin(1);
    opf::launch_zsynth32(d, g.ds, g.pz, g.W6f, g.Z6f, st);
    r->end();
    r->begin(2);
    opf::launch_product32(d, g.ds, g.pth, g.Z6f, g.ZNf, st);
    r->end();
    r->begin(3);
    opf::launch_zanalysis32(d, g.ds, g.pz, g.ZNf, g.Nlin, Nout, st);
    r->end();
    return;
  }
  r->begin(1);
  opf::launch_zsynth(d, g.ds, g.pz, g.W6, g.Z6, st);
  r->end();
  r->begin(2);
  opf::launch_product(d, g.ds, g.pth, g.Z6, g.ZN, st);
  r->end();
  r->begin(3);
  opf::launch_zanalysis(d, g.ds, g.pz, g.ZN, Nout, st);
  r->end();
}

// FP64 steps fuse the curl into the solve: the solve blocks leave the curl
// of their output in W6 for the next nonlinear evaluation (measured: FP64
// medium step 441 -> 394 us).  Mixed-precision steps keep the separate split
// curl: there the fused form cost the solve about as much as the curl launch
// it saved.
bool fused_curl(const Runner* r) { return r->precision == 0; }

// Solve pass into Uout (and, fused, the curl of Uout into W6).
void enqueue_solve(Runner* r, const Group& g, const double2* Na, const double2* Nb, double wa,
                   double wb, double2* Uout) {
  opf::SolveArgs a{g.U, Na, Nb, wa, wb, Uout, g.beta_p};
  if (fused_curl(r)) {
    a.curl = 1;
    a.W6 = (void*)g.W6;
  }
  r->begin(4);
  opf::launch_solve(g.d, g.ds, a, g.nJ, r->st());
  r->end();
}

// Side streams and fork/join events for groups 1..n-1 (created once).
bool ensure_side_streams(Runner* r) {
  const size_t need = r->groups.size() - 1;
  if (!r->fork_ev && cudaEventCreateWithFlags(&r->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
    r->fork_ev = nullptr;
    return false;
  }
  while (r->side.size() < need) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(s);
      return false;
    }
    r->side.push_back(s);
    r->join_ev.push_back(e);
  }
  return true;
}

// One predictor-corrector step (section 2) of every trajectory of every
// group: predictor with N_j, then n_corr corrector passes with
// c N^q + (1 - c) N_j, each solved from u_j.  The groups are independent:
// with more than one, groups 1.. run on side streams forked from the main
// stream and joined back (parallel graph branches), so that one group's
// FP64-bound solves overlap another's transforms.  Per-kernel timing
// (timing 1) keeps them in one stream.
void enqueue_step(Runner* r) {
  const size_t ng = r->groups.size();
  const bool fork = ng > 1 && r->timing != 1 && ensure_side_streams(r);
  if (fork) cudaEventRecord(r->fork_ev, r->stream);
  for (size_t i = 0; i < ng; ++i) {
    Group* g = r->groups[i];
    r->cur = nullptr;
    if (fork && i > 0) {
      r->cur = r->side[i - 1];
      cudaStreamWaitEvent(r->cur, r->fork_ev, 0);
    }
    const double c = g->d.c;
    if (g->d.cfl) cudaMemsetAsync(g->cfl, 0, sizeof(double), r->st());
    // fused: W6 holds the curl of U at the start of a step (runner_step) and
    // the solves leave the curl of their output
    const bool curl = !fused_curl(r);
    enqueue_nonlinear(r, *g, g->U, g->Nj, curl);
    enqueue_solve(r, *g, g->Nj, nullptr, 1.0, 0.0, g->U1);
    if (r->n_corr == 0)  // predictor only: its output (3F per trajectory) is the new state
      cudaMemcpy2DAsync(g->U, g->sstride, g->U1, g->sstride, 3 * (size_t)g->d.F * sizeof(double2), g->d.B,
                        cudaMemcpyDeviceToDevice, r->st());
    for (int q = 0; q < r->n_corr; ++q) {
      enqueue_nonlinear(r, *g, g->U1, g->Nq, curl);
      enqueue_solve(r, *g, g->Nq, g->Nj, c, 1.0 - c, q == r->n_corr - 1 ? g->U : g->U1);
    }
    if (fork && i > 0) cudaEventRecord(r->join_ev[i - 1], r->cur);
  }
  r->cur = nullptr;
  if (fork)
    for (size_t i = 1; i < ng; ++i) cudaStreamWaitEvent(r->stream, r->join_ev[i - 1], 0);
}

int harvest_timing(Runner* r) {
  if (!r->timing) return OPF_OK;
  for (int i = 0; i < r->nslots; ++i) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, r->ev[i][0], r->ev[i][1]));
    r->tot_ms[r->slot_name[i]] += ms;
    r->tot_n[r->slot_name[i]] += 1;
  }
  return OPF_OK;
}

// ---- autotuner: per group, time each transform kernel and the solve over
// the launch shapes whose shared memory fits, on the group's current state
// (every timed kernel is idempotent: it rewrites only scratch buffers).
template <typename F>
float time_launch(Runner* r, F launch) {
  launch();
  cudaEventRecord(r->ev[0][0], r->stream);
  for (int rep = 0; rep < 3; ++rep) launch();
  cudaEventRecord(r->ev[0][1], r->stream);
  cudaEventSynchronize(r->ev[0][1]);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, r->ev[0][0], r->ev[0][1]);
  return ms / 3.f;
}

int tune_group(Runner* r, Group* g) {
  g->w6_valid = false;  // the timed launches overwrite the work buffers
  opf::Dims& d = g->d;
  int dev = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t vb = r->precision == 1 ? sizeof(float2) : sizeof(double2);
  const bool mixed = r->precision == 1;
  cudaStream_t st = r->stream;
  // valid inputs for every stage: one nonlinear evaluation of the state
  enqueue_nonlinear(r, *g, g->U, g->Nj);
  const int cand[5] = {1, 2, 4, 8, 16};
  float best = 1e30f;
  int pick = d.mcz;
  for (int c : cand) {
    if (c > d.M || opf::zsynth_smem(d, c, vb) > (size_t)optin) continue;
    d.mcz = c;
    const float t = time_launch(r, [&] {
      if (mixed) opf::launch_zsynth32(d, g->ds, g->pz, g->W6f, g->Z6f, st);
      else opf::launch_zsynth(d, g->ds, g->pz, g->W6, g->Z6, st);
    });
    if (t < best) best = t, pick = c;
  }
  d.mcz = pick;
  best = 1e30f;
  pick = d.zc;
  for (int c : cand) {
    if (c > d.nz || opf::product_smem(d, c, vb) > (size_t)optin) continue;
    d.zc = c;
    const float t = time_launch(r, [&] {
      if (mixed) opf::launch_product32(d, g->ds, g->pth, g->Z6f, g->ZNf, st);
      else opf::launch_product(d, g->ds, g->pth, g->Z6, g->ZN, st);
    });
    if (t < best) best = t, pick = c;
  }
  d.zc = pick;
  best = 1e30f;
  pick = d.mca;
  for (int c : cand) {
    if (c > d.M || opf::zanalysis_smem(d, c, vb) > (size_t)optin) continue;
    d.mca = c;
    const float t = time_launch(r, [&] {
      if (mixed) opf::launch_zanalysis32(d, g->ds, g->pz, g->ZNf, g->Nlin, g->Nq, st);
      else opf::launch_zanalysis(d, g->ds, g->pz, g->ZN, g->Nq, st);
    });
    if (t < best) best = t, pick = c;
  }
  d.mca = pick;
  if (mixed) {  // the three transforms as they stand, against the fused launch per cluster size
    d.fused = 0;
    best = time_launch(r, [&] {
      opf::launch_zsynth32(d, g->ds, g->pz, g->W6f, g->Z6f, st);
      opf::launch_product32(d, g->ds, g->pth, g->Z6f, g->ZNf, st);
      opf::launch_zanalysis32(d, g->ds, g->pz, g->ZNf, g->Nlin, g->Nq, st);
    });
    pick = 0;
    for (int C : {2, 4, 8}) {
      d.fused = C;
      if (opf::fused32_cluster(d) != C) continue;
      const float t = time_launch(r, [&] { opf::launch_nl_fused32(d, g->ds, g->W6f, g->Nlin, g->Nq, st); });
      if (t < best) best = t, pick = C;
    }
    d.fused = pick;
  }
  // the split solve (4-mode tiles only) changes the rounding order of the
  // substitution, so the tuner keeps it and its tile: launch shapes alone are
  // tuned, never the arithmetic
  best = 1e30f;
  pick = d.spike ? 4 : 0;
  for (int T : {4, 8, 16}) {
    if (d.spike) break;
    if (opf::solve_smem_bytes(d.N, T) > (size_t)optin) continue;
    d.tile = T;
    opf::SolveArgs a{g->U, g->Nj, nullptr, 1.0, 0.0, g->U1, g->beta_p};
    const float t = time_launch(r, [&] { opf::launch_solve(d, g->ds, a, g->nJ, st); });
    if (t < best) best = t, pick = T;
  }
  d.tile = pick;
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());
  return OPF_OK;
}

// CFL control (single trajectory): dt = min(dt_max, C / max(|u|/spacing)),
// changed only when it must drop or could rise by more than 10 %; the
// dt-dependent operators are then rebuilt in place.
int cfl_update(Runner* r) {
  for (Group* g : r->groups) {
    if (!g->d.cfl || g->d.B != 1) continue;
    double c = 0.0;
    CU(cudaMemcpyAsync(&c, g->cfl, sizeof(double), cudaMemcpyDeviceToHost, r->stream));
    CU(cudaStreamSynchronize(r->stream));
    if (!(c > 0.0) || !std::isfinite(c)) continue;
    const double target = std::min(r->dt_max, r->cfl_C / c);
    const double cur = g->dt[0];
    if (target < cur || target > 1.1 * cur) {
      g->dt[0] = target;
      g->d.dt = target;
      int rc = group_fill_setups(g, false);
      if (rc) return rc;
    }
  }
  return OPF_OK;
}

int runner_step(Runner* r, int n) {
  if (n < 0) return fail(OPF_EINVAL, "step: n < 0");
  if (r->autotune == 1) {
    const int timing = r->timing;
    r->timing = 0;
    for (Group* g : r->groups) {
      int rc = tune_group(r, g);
      if (rc) return rc;
    }
    r->timing = timing;
    r->autotune = 2;  // tuned
    r->drop_graph();
  }
  for (int s = 0; s < n; ++s) {
    r->nslots = 0;
    for (Group* g : r->groups)
      if (fused_curl(r) && !g->w6_valid) {  // the step graph starts from the curl of U (untimed)
        enqueue_curl(r, *g, g->U, false);
        g->w6_valid = true;
      }
    if (r->use_graph) {
      if (!r->gexec) {
        cudaGraph_t gr;
        CU(cudaStreamBeginCapture(r->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_step(r);
        cudaError_t e = cudaStreamEndCapture(r->stream, &gr);
        if (e != cudaSuccess) return fail(OPF_ECUDA, std::string("stream capture: ") + cudaGetErrorString(e));
        r->graph_nslots = r->nslots;
        e = cudaGraphInstantiate(&r->gexec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
          r->gexec = nullptr;
          return fail(OPF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
      }
      CU(cudaGraphLaunch(r->gexec, r->stream));
      r->nslots = r->graph_nslots;  // event nodes captured with the graph
    } else {
      enqueue_step(r);
    }
    if (r->timing) {
      CU(cudaStreamSynchronize(r->stream));
      int rc = harvest_timing(r);
      if (rc) return rc;
    }
    for (Group* g : r->groups)
      for (int b = 0; b < g->d.B; ++b) g->time[b] += g->dt[b];
    if (r->cfl_C > 0.0) {
      int rc = cfl_update(r);
      if (rc) return rc;
    }
  }
  CU(cudaStreamSynchronize(r->stream));
  CU(cudaGetLastError());
  return OPF_OK;
}

int runner_option(Runner* r, const char* key, double v) {
  if (!key) return fail(OPF_EINVAL, "set_option: NULL key");
  for (Group* g : r->groups) g->w6_valid = false;  // precision / frame rotation change W6
  if (!strcmp(key, "precision")) {
    if (v != 0.0 && v != 1.0) return fail(OPF_EINVAL, "precision: 0 (FP64) or 1 (mixed)");
    r->precision = (int)v;
  } else if (!strcmp(key, "n_corr")) {
    if (!(v >= 0 && v <= 16 && v == std::floor(v))) return fail(OPF_EINVAL, "n_corr: 0..16");
    r->n_corr = (int)v;
  } else if (!strcmp(key, "graph")) {
    if (v != 0.0 && v != 1.0) return fail(OPF_EINVAL, "graph: 0 or 1");
    r->use_graph = (int)v;
  } else if (!strcmp(key, "timing")) {
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(OPF_EINVAL, "timing: 0, 1 or 2");
    if ((int)v != r->timing) r->drop_graph();  // the event nodes are part of the graph
    r->timing = (int)v;
  } else if (!strcmp(key, "timed_kernel")) {
    if (!(v >= 0 && v <= 5 && v == std::floor(v))) return fail(OPF_EINVAL, "timed_kernel: 0..5");
    r->timed_kernel = (int)v;
  } else if (!strcmp(key, "autotune")) {
    if (v != 0.0 && v != 1.0) return fail(OPF_EINVAL, "autotune: 0 or 1");
    r->autotune = (int)v;
  } else if (!strcmp(key, "rot_x") || !strcmp(key, "rot_y") || !strcmp(key, "rot_z")) {
    // frame rotation, shared by every trajectory (all groups)
    if (!std::isfinite(v)) return fail(OPF_EINVAL, "rotation: finite value");
    for (Group* g : r->groups) {
      const opf::Dims& d = g->d;
      const double x = key[4] == 'x' ? v : d.rot_x, y = key[4] == 'y' ? v : d.rot_y;
      if ((x != 0.0 || y != 0.0) && d.m_p != 1)
        return fail(OPF_EINVAL, "rotation about a transverse axis needs m_p = 1 (it couples m to m +- 1)");
    }
    for (Group* g : r->groups) {
      opf::Dims& d = g->d;
      (key[4] == 'x' ? d.rot_x : key[4] == 'y' ? d.rot_y : d.rot_z) = v;
      d.rotate = (d.rot_x != 0.0 || d.rot_y != 0.0 || d.rot_z != 0.0) ? 1 : 0;
    }
  } else if (!strcmp(key, "spike")) {
    if (v != 0.0 && v != 1.0) return fail(OPF_EINVAL, "spike: 0 or 1");
    for (Group* g : r->groups) g->d.spike = (v != 0.0 && g->spike_built) ? 1 : 0;
  } else if (!strcmp(key, "fused")) {
    if (v != 0.0 && v != 1.0 && v != 2.0 && v != 4.0 && v != 8.0)
      return fail(OPF_EINVAL, "fused: 0 (off), 1 (cluster size chosen), 2, 4 or 8 (cluster size)");
    for (Group* g : r->groups) g->d.fused = (int)v;
  } else if (!strcmp(key, "pdl")) {
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(OPF_EINVAL, "pdl: 0, 1 or 2");
    for (Group* g : r->groups) g->d.pdl = (int)v;
  } else if (!strcmp(key, "tile")) {
    if (v != 0.0 && v != 4.0 && v != 8.0 && v != 16.0)
      return fail(OPF_EINVAL, "tile: 0 (heuristic), 4, 8 or 16 modes per solve block");
    int dev = 0, optin = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (Group* g : r->groups)
      if (v != 0.0 && opf::solve_smem_bytes(g->d.N, (int)v) > (size_t)optin)
        return fail(OPF_EINVAL, "tile: the solve block of this size does not fit in shared memory");
    for (Group* g : r->groups) g->d.tile = (int)v;
  } else {
    return fail(OPF_EINVAL, std::string("unknown option ") + key);
  }
  r->drop_graph();
  return OPF_OK;
}

int runner_get_option(Runner* r, const char* key, double* v) {
  if (!key || !v) return fail(OPF_EINVAL, "get_option: NULL argument");
  if (!strcmp(key, "precision")) *v = r->precision;
  else if (!strcmp(key, "n_corr")) *v = r->n_corr;
  else if (!strcmp(key, "graph")) *v = r->use_graph;
  else if (!strcmp(key, "timing")) *v = r->timing;
  else if (!strcmp(key, "timed_kernel")) *v = r->timed_kernel;
  else if (!strcmp(key, "autotune")) *v = r->autotune;
  else if (!strcmp(key, "tile")) *v = r->groups.empty() ? 0 : r->groups[0]->d.tile;
  else if (!strcmp(key, "pdl")) *v = r->groups.empty() ? 0 : r->groups[0]->d.pdl;
  else if (!strcmp(key, "fused")) *v = r->groups.empty() ? 0 : opf::fused32_cluster(r->groups[0]->d);
  else if (!strcmp(key, "spike")) *v = r->groups.empty() ? 0 : r->groups[0]->d.spike;
  else if (!strcmp(key, "rot_x")) *v = r->groups.empty() ? 0 : r->groups[0]->d.rot_x;
  else if (!strcmp(key, "rot_y")) *v = r->groups.empty() ? 0 : r->groups[0]->d.rot_y;
  else if (!strcmp(key, "rot_z")) *v = r->groups.empty() ? 0 : r->groups[0]->d.rot_z;
  else if (!strcmp(key, "mcz")) *v = r->groups.empty() ? 0 : r->groups[0]->d.mcz;
  else if (!strcmp(key, "mca")) *v = r->groups.empty() ? 0 : r->groups[0]->d.mca;
  else if (!strcmp(key, "zc")) *v = r->groups.empty() ? 0 : r->groups[0]->d.zc;
  else return fail(OPF_EINVAL, std::string("unknown option ") + key);
  return OPF_OK;
}

int runner_times(Runner* r, int cap, int* count, const char** names, double* total_ms, int* launches,
                 int reset) {
  if (!count) return fail(OPF_EINVAL, "NULL count");
  int c = 0;
  for (int i = 0; i < kNumNames && c < cap; ++i) {
    if (names) names[c] = kNames[i];
    if (total_ms) total_ms[c] = r->tot_ms[i];
    if (launches) launches[c] = r->tot_n[i];
    ++c;
  }
  *count = c;
  if (reset)
    for (int i = 0; i < kNumNames; ++i) {
      r->tot_ms[i] = 0;
      r->tot_n[i] = 0;
    }
  return OPF_OK;
}

// ---- per-trajectory state transfer and diagnostics
int traj_state_from_abi(Group* g, int b, cudaStream_t st, bool note = true);

// The words a set_state reads back from the trajectory's flag slot: a
// non-finite coefficient was seen; the m = 0 asymmetry and magnitude maxima of
// the layout conversion (upper 32 bits of non-negative doubles).
struct SetFlags {
  int nan;
  unsigned asym_hi, amp_hi;
};

// Leaves a note for opf_last_error() when the m = 0 coefficients were not
// Hermitian to 1e-12 of the largest of them (the state is projected all the
// same, section 2: the fields are real).
void note_asymmetry(const SetFlags& f) {
  auto value = [](unsigned hi) {
    const unsigned long long bits = (unsigned long long)hi << 32;
    double v;
    std::memcpy(&v, &bits, sizeof v);
    return v;
  };
  const double asym = value(f.asym_hi), amp = value(f.amp_hi);
  if (asym > 1e-12 * amp) {
    char msg[160];
    std::snprintf(msg, sizeof msg,
                  "set_state: m = 0 coefficients not Hermitian (max |A(k,0) - conj A(-k,0)| = %.3g of the "
                  "largest); projected",
                  asym / amp);
    opf::set_last_error(msg);
  }
}

int traj_set_state_device(Group* g, int b, const double* d_coeffs, cudaStream_t st) {
  const size_t bytes = 3 * (size_t)g->d.F * sizeof(double2);
  CU(cudaMemcpyAsync(g->at(g->abi, b), d_coeffs, bytes, cudaMemcpyDeviceToDevice, st));
  return traj_state_from_abi(g, b, st);
}

// The trajectory's staging copy (abi) into its state: a NaN check, then the
// layout conversion (with the Hermitian projection and beta reset), which
// the device skips when the check found a non-finite value -- so the state
// is unchanged on OPF_ENAN -- and one synchronisation for both.  note: leave
// the m = 0 asymmetry note (note_asymmetry) where there is one.
int traj_state_from_abi(Group* g, int b, cudaStream_t st, bool note) {
  const opf::Dims d = g->single(b);
  double2* abi = g->at(g->abi, b);
  int* flag = g->at(g->flag, b);
  opf::launch_nan_check((const double*)abi, 6 * d.F, flag, st);
  CU(cudaMemsetAsync(flag + 1, 0, 2 * sizeof(unsigned), st));
  opf::launch_abi_to_internal(d, abi, g->at(g->U, b), st, flag, g->at(g->beta_p, b), nullptr, (unsigned*)(flag + 1));
  SetFlags hf{};
  CU(cudaMemcpyAsync(&hf, flag, sizeof hf, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());
  if (hf.nan) return fail(OPF_ENAN, "set_state: non-finite coefficient; state unchanged");
  if (note) note_asymmetry(hf);
  g->w6_valid = false;
  return OPF_OK;
}

// The device address of a host buffer the GPU can read and write directly --
// pinned memory (cudaHostAlloc, cudaMallocHost, cudaHostRegister) is mapped
// under unified addressing -- else nullptr (pageable memory: copies instead).
const void* device_view(const void* host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

int traj_set_state_host(Group* g, int b, const double* coeffs, cudaStream_t st, bool note = true) {
  const opf::Dims d = g->single(b);
  if (const void* dv = device_view(coeffs)) {
    // pinned: the conversion reads the buffer itself (one pass, with the NaN
    // check) into scratch, which replaces the state only if every value was
    // finite; one synchronisation
    int* flag = g->at(g->flag, b);
    double2* tmp = g->at(g->tmpU, b);
    CU(cudaMemsetAsync(flag, 0, sizeof(SetFlags), st));
    opf::launch_abi_to_internal(d, (const double2*)dv, tmp, st, nullptr, nullptr, flag, (unsigned*)(flag + 1));
    opf::launch_copy_unless(tmp, g->at(g->U, b), 3 * (long)d.F, flag, g->at(g->beta_p, b), st);
    SetFlags hf{};
    CU(cudaMemcpyAsync(&hf, flag, sizeof hf, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    CU(cudaGetLastError());
    if (hf.nan) return fail(OPF_ENAN, "set_state: non-finite coefficient; state unchanged");
    if (note) note_asymmetry(hf);
    g->w6_valid = false;
    return OPF_OK;
  }
  CU(cudaMemcpyAsync(g->at(g->abi, b), coeffs, 3 * (size_t)d.F * sizeof(double2), cudaMemcpyHostToDevice, st));
  return traj_state_from_abi(g, b, st, note);
}

int traj_get_state(Group* g, int b, double* out, bool host, cudaStream_t st) {
  const opf::Dims d = g->single(b);
  double2* abi = g->at(g->abi, b);
  void* dv = host ? const_cast<void*>(device_view(out)) : nullptr;  // pinned: written by the kernel itself
  opf::launch_internal_to_abi(d, g->at(g->U, b), dv ? (double2*)dv : host ? abi : (double2*)out, 1, st);
  if (host && !dv)
    CU(cudaMemcpyAsync(out, abi, 3 * (size_t)d.F * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());
  return OPF_OK;
}

int traj_energy(Group* g, int b, double out[3], cudaStream_t st) {
  const opf::Dims d = g->single(b);
  const opf::DevSetup s = g->setup_of(b);
  double2* U = g->at(g->U, b);
  double2* W6 = g->at(g->W6, b);
  g->w6_valid = false;  // FP64 curl of this trajectory only
  opf::launch_curl(d, s, U, W6, st);
  opf::launch_energy(d, s, U, W6, g->at(g->beta_p, b), g->at(g->partial, b), g->nblk_energy,
                     g->at(g->out3, b), st);
  CU(cudaMemcpyAsync(out, g->at(g->out3, b), 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());
  if (!std::isfinite(out[0]) || !std::isfinite(out[1]) || !std::isfinite(out[2]))
    return fail(OPF_ENAN, "energy: non-finite state");
  return OPF_OK;
}

int traj_beta(Group* g, int b, double* beta, cudaStream_t st) {
  double bp = 0.0;
  CU(cudaMemcpyAsync(&bp, g->at(g->beta_p, b), sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *beta = bp * g->Re[b] / 4.0;
  return OPF_OK;
}

}  // namespace

// ====================================================================== handles
struct opf_ctx {
  Group g;
  Runner run;
  double2* forcing = nullptr;  // constant body force, internal +- layout (opf_set_forcing)
};

struct opf_ens {
  std::vector<Group> groups;
  std::vector<std::pair<int, int>> where;  // trajectory -> (group, index in group)
  Runner run;
};

namespace {
int check_handle(const void* h) { return h ? OPF_OK : fail(OPF_EINVAL, "NULL handle"); }
}  // namespace

extern "C" {

const char* opf_last_error(void) { return g_err.c_str(); }

opf_t* opf_create(int N, int K, int M, int m_p, double alpha, double Re, double dt) {
  return opf_create_mesh(N, K, M, m_p, alpha, Re, dt, nullptr);
}

opf_t* opf_create_mesh(int N, int K, int M, int m_p, double alpha, double Re, double dt, const double* r) {
  opf_ctx* h = new opf_ctx();
  if (r && N > 0) h->g.mesh.assign(r, r + N);
  int rc = group_build(&h->g, N, K, M, m_p, alpha, 1, &Re, &dt);
  if (rc == OPF_OK) rc = runner_init(&h->run);
  if (rc == OPF_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = fail(OPF_ECUDA, cudaGetErrorString(e));
  }
  if (rc != OPF_OK) {
    std::string keep = "opf_create: " + g_err;
    group_free(&h->g);
    runner_free(&h->run);
    delete h;
    g_err = keep;
    return nullptr;
  }
  h->run.groups = {&h->g};
  return h;
}

void opf_destroy(opf_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->run.stream);
  runner_free(&h->run);
  group_free(&h->g);
  if (h->forcing) cudaFree(h->forcing);
  delete h;
}

int opf_set_forcing(opf_t* h, const double* coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  CU(cudaStreamSynchronize(h->run.stream));
  h->run.drop_graph();
  if (!coeffs) {
    h->g.d.forcing = nullptr;
    return OPF_OK;
  }
  const size_t bytes = 3 * (size_t)h->g.d.F * sizeof(double2);
  if (!h->forcing) CU(cudaMalloc((void**)&h->forcing, bytes));
  double2* abi = h->g.at(h->g.abi, 0);  // staging in the ABI layout
  CU(cudaMemcpyAsync(abi, coeffs, bytes, cudaMemcpyHostToDevice, h->run.stream));
  opf::Dims d1 = h->g.single(0);
  opf::launch_abi_to_internal(d1, abi, h->forcing, h->run.stream);
  CU(cudaStreamSynchronize(h->run.stream));
  CU(cudaGetLastError());
  h->g.d.forcing = h->forcing;
  return OPF_OK;
}

int opf_set_state_device(opf_t* h, const double* d_coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!d_coeffs) return fail(OPF_EINVAL, "opf_set_state: NULL buffer");
  g_err.clear();
  return traj_set_state_device(&h->g, 0, d_coeffs, h->run.stream);
}

int opf_set_state(opf_t* h, const double* coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!coeffs) return fail(OPF_EINVAL, "opf_set_state: NULL buffer");
  g_err.clear();
  return traj_set_state_host(&h->g, 0, coeffs, h->run.stream);
}

int opf_get_state_device(opf_t* h, double* d_coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!d_coeffs) return fail(OPF_EINVAL, "opf_get_state: NULL buffer");
  return traj_get_state(&h->g, 0, d_coeffs, false, h->run.stream);
}

int opf_get_state(opf_t* h, double* coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!coeffs) return fail(OPF_EINVAL, "opf_get_state: NULL buffer");
  return traj_get_state(&h->g, 0, coeffs, true, h->run.stream);
}

int opf_step(opf_t* h, int n) {
  if (check_handle(h)) return OPF_EINVAL;
  return runner_step(&h->run, n);
}

int opf_energy(opf_t* h, double out[3]) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!out) return fail(OPF_EINVAL, "opf_energy: NULL out");
  return traj_energy(&h->g, 0, out, h->run.stream);
}

int opf_wall_residual(opf_t* h, double out[2]) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!out) return fail(OPF_EINVAL, "opf_wall_residual: NULL out");
  opf::launch_wall(h->g.single(0), h->g.ds, h->g.U, h->g.out2, h->run.stream);
  CU(cudaMemcpyAsync(out, h->g.out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->run.stream));
  CU(cudaStreamSynchronize(h->run.stream));
  CU(cudaGetLastError());
  return OPF_OK;
}

int opf_nonlinear(opf_t* h, const double* coeffs, double* out) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!coeffs || !out) return fail(OPF_EINVAL, "opf_nonlinear: NULL buffer");
  Group& g = h->g;
  cudaStream_t st = h->run.stream;
  const size_t bytes = 3 * (size_t)g.d.F * sizeof(double2);
  CU(cudaMemcpyAsync(g.abi, coeffs, bytes, cudaMemcpyHostToDevice, st));
  opf::launch_abi_to_internal(g.d, g.abi, g.tmpU, st);
  const int timing = h->run.timing;
  h->run.timing = 0;
  g.w6_valid = false;  // W6 takes the curl of the given state
  enqueue_nonlinear(&h->run, g, g.tmpU, g.Nq);
  h->run.timing = timing;
  opf::launch_internal_to_abi(g.d, g.Nq, g.abi, 1, st);
  CU(cudaMemcpyAsync(out, g.abi, bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());
  return OPF_OK;
}

int opf_set_option(opf_t* h, const char* key, double v) {
  if (check_handle(h)) return OPF_EINVAL;
  if (key && !strcmp(key, "cfl")) {  // CFL number C; 0 switches control off
    if (!(v >= 0.0 && v <= 10.0)) return fail(OPF_EINVAL, "cfl: 0 (off) .. 10");
    h->run.cfl_C = v;
    if (h->run.dt_max <= 0.0) h->run.dt_max = h->g.dt[0];
    h->g.d.cfl = v > 0.0 ? h->g.cfl : nullptr;
    h->g.d.rinv_cfl = h->g.ds.rinv;
    h->run.drop_graph();
    return OPF_OK;
  }
  if (key && !strcmp(key, "dt_max")) {
    if (!(v > 0.0)) return fail(OPF_EINVAL, "dt_max: > 0");
    h->run.dt_max = v;
    return OPF_OK;
  }
  if (key && !strcmp(key, "dt")) {  // set the time step; dt-dependent operators are refactored
    if (!(v > 0.0) || !std::isfinite(v)) return fail(OPF_EINVAL, "dt: > 0");
    if (v != h->g.dt[0]) {
      CU(cudaStreamSynchronize(h->run.stream));
      h->g.dt[0] = v;
      h->g.d.dt = v;
      return group_fill_setups(&h->g, false);
    }
    return OPF_OK;
  }
  return runner_option(&h->run, key, v);
}

int opf_get_option(opf_t* h, const char* key, double* v) {
  if (check_handle(h)) return OPF_EINVAL;
  if (key && v && !strcmp(key, "cfl")) {
    *v = h->run.cfl_C;
    return OPF_OK;
  }
  if (key && v && !strcmp(key, "dt_max")) {
    *v = h->run.dt_max > 0.0 ? h->run.dt_max : h->g.dt[0];
    return OPF_OK;
  }
  if (key && v && !strcmp(key, "cfl_number")) {  // max |u| dt / spacing of the last step
    double c = 0.0;
    CU(cudaMemcpy(&c, h->g.cfl, sizeof(double), cudaMemcpyDeviceToHost));
    *v = c * h->g.dt[0];
    return OPF_OK;
  }
  return runner_get_option(&h->run, key, v);
}

int opf_get_dt(opf_t* h, double* dt) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!dt) return fail(OPF_EINVAL, "NULL out");
  *dt = h->g.dt[0];
  return OPF_OK;
}

int opf_get_time(opf_t* h, double* t) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!t) return fail(OPF_EINVAL, "NULL out");
  *t = h->g.time[0];
  return OPF_OK;
}

int opf_get_beta(opf_t* h, double* beta) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!beta) return fail(OPF_EINVAL, "NULL out");
  return traj_beta(&h->g, 0, beta, h->run.stream);
}

int opf_set_stream(opf_t* h, void* stream) {
  if (check_handle(h)) return OPF_EINVAL;
  CU(cudaStreamSynchronize(h->run.stream));
  h->run.stream = stream ? (cudaStream_t)stream : h->run.own;
  return OPF_OK;
}

int opf_kernel_times(opf_t* h, int cap, int* count, const char** names, double* total_ms,
                     int* launches, int reset) {
  if (check_handle(h)) return OPF_EINVAL;
  return runner_times(&h->run, cap, count, names, total_ms, launches, reset);
}

// ---------------------------------------------------------------- ensembles
opf_ens_t* opf_ens_create(int count, const int* N, const int* K, const int* M, const int* m_p,
                          const double* alpha, const double* Re, const double* dt) {
  if (count < 1 || !N || !K || !M || !m_p || !alpha || !Re || !dt) {
    fail(OPF_EINVAL, "opf_ens_create: need count >= 1 and non-NULL arrays");
    return nullptr;
  }
  // group trajectories by shape, keeping their order inside each group
  std::map<std::tuple<int, int, int, int, double>, std::vector<int>> by_shape;
  std::vector<std::tuple<int, int, int, int, double>> order;
  for (int i = 0; i < count; ++i) {
    auto key = std::make_tuple(N[i], K[i], M[i], m_p[i], alpha[i]);
    if (!by_shape.count(key)) order.push_back(key);
    by_shape[key].push_back(i);
  }
  opf_ens* e = new opf_ens();
  e->groups.resize(order.size());
  e->where.assign(count, {0, 0});
  int rc = OPF_OK;
  for (size_t gi = 0; gi < order.size() && rc == OPF_OK; ++gi) {
    const auto& idx = by_shape[order[gi]];
    std::vector<double> re, tt;
    for (int i : idx) {
      re.push_back(Re[i]);
      tt.push_back(dt[i]);
    }
    const auto& k = order[gi];
    rc = group_build(&e->groups[gi], std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                     std::get<4>(k), (int)idx.size(), re.data(), tt.data());
    for (size_t b = 0; b < idx.size(); ++b) e->where[idx[b]] = {(int)gi, (int)b};
  }
  if (rc == OPF_OK) rc = runner_init(&e->run);
  if (rc != OPF_OK) {
    std::string keep = "opf_ens_create: " + g_err;
    for (Group& g : e->groups) group_free(&g);
    runner_free(&e->run);
    delete e;
    g_err = keep;
    return nullptr;
  }
  for (Group& g : e->groups) e->run.groups.push_back(&g);
  return e;
}

void opf_ens_destroy(opf_ens_t* e) {
  if (!e) return;
  cudaStreamSynchronize(e->run.stream);
  runner_free(&e->run);
  for (Group& g : e->groups) group_free(&g);
  delete e;
}

namespace {
int ens_traj(opf_ens_t* e, int i, Group** g, int* b) {
  if (!e) return fail(OPF_EINVAL, "NULL ensemble");
  if (i < 0 || i >= (int)e->where.size()) return fail(OPF_EINVAL, "trajectory index out of range");
  *g = &e->groups[e->where[i].first];
  *b = e->where[i].second;
  return OPF_OK;
}
}  // namespace

int opf_ens_count(opf_ens_t* e, int* count) {
  if (check_handle(e) || !count) return fail(OPF_EINVAL, "NULL argument");
  *count = (int)e->where.size();
  return OPF_OK;
}

int opf_ens_set_state(opf_ens_t* e, int i, const double* coeffs) {
  Group* g;
  int b;
  if (ens_traj(e, i, &g, &b)) return OPF_EINVAL;
  if (!coeffs) return fail(OPF_EINVAL, "opf_ens_set_state: NULL buffer");
  g_err.clear();
  return traj_set_state_host(g, b, coeffs, e->run.stream);
}

int opf_ens_get_state(opf_ens_t* e, int i, double* coeffs) {
  Group* g;
  int b;
  if (ens_traj(e, i, &g, &b)) return OPF_EINVAL;
  if (!coeffs) return fail(OPF_EINVAL, "opf_ens_get_state: NULL buffer");
  return traj_get_state(g, b, coeffs, true, e->run.stream);
}

int opf_ens_set_state_device(opf_ens_t* e, int i, const double* d_coeffs) {
  Group* g;
  int b;
  if (ens_traj(e, i, &g, &b)) return OPF_EINVAL;
  if (!d_coeffs) return fail(OPF_EINVAL, "opf_ens_set_state_device: NULL buffer");
  g_err.clear();
  return traj_set_state_device(g, b, d_coeffs, e->run.stream);
}

int opf_ens_get_state_device(opf_ens_t* e, int i, double* d_coeffs) {
  Group* g;
  int b;
  if (ens_traj(e, i, &g, &b)) return OPF_EINVAL;
  if (!d_coeffs) return fail(OPF_EINVAL, "opf_ens_get_state_device: NULL buffer");
  return traj_get_state(g, b, d_coeffs, false, e->run.stream);
}

int opf_ens_step(opf_ens_t* e, int n) {
  if (check_handle(e)) return OPF_EINVAL;
  return runner_step(&e->run, n);
}

int opf_ens_energy(opf_ens_t* e, int i, double out[3]) {
  Group* g;
  int b;
  if (ens_traj(e, i, &g, &b)) return OPF_EINVAL;
  if (!out) return fail(OPF_EINVAL, "opf_ens_energy: NULL out");
  return traj_energy(g, b, out, e->run.stream);
}

int opf_ens_get_time(opf_ens_t* e, int i, double* t) {
  Group* g;
  int b;
  if (ens_traj(e, i, &g, &b)) return OPF_EINVAL;
  if (!t) return fail(OPF_EINVAL, "NULL out");
  *t = g->time[b];
  return OPF_OK;
}

int opf_ens_set_option(opf_ens_t* e, const char* key, double v) {
  if (check_handle(e)) return OPF_EINVAL;
  return runner_option(&e->run, key, v);
}

int opf_ens_set_stream(opf_ens_t* e, void* stream) {
  if (check_handle(e)) return OPF_EINVAL;
  CU(cudaStreamSynchronize(e->run.stream));
  e->run.stream = stream ? (cudaStream_t)stream : e->run.own;
  e->run.drop_graph();
  return OPF_OK;
}

int opf_ens_kernel_times(opf_ens_t* e, int cap, int* count, const char** names, double* total_ms,
                         int* launches, int reset) {
  if (check_handle(e)) return OPF_EINVAL;
  return runner_times(&e->run, cap, count, names, total_ms, launches, reset);
}

// ---------------------------------------------------------------- host-only
int opf_setup_query(int N, int K, int M, int m_p, double alpha, double Re, double dt,
                    const char* what, double* out, long cap, long* len) {
  return opf_setup_query_mesh(N, K, M, m_p, alpha, Re, dt, nullptr, what, out, cap, len);
}

int opf_setup_query_mesh(int N, int K, int M, int m_p, double alpha, double Re, double dt, const double* r,
                         const char* what, double* out, long cap, long* len) {
  if (N < 9 || K < 1 || M < 1 || m_p < 1 || !(alpha > 0) || !(Re > 0) || !(dt > 0) || !what || !len)
    return fail(OPF_EINVAL, "opf_setup_query: bad arguments");
  opf::Setup s;
  if (r) s.r_user.assign(r, r + N);
  s.N = N;
  s.K = K;
  s.M = M;
  s.m_p = m_p;
  s.alpha = alpha;
  s.Re = Re;
  s.dt = dt;
  s.c = 0.5;
  const char* split_arrays[] = {"luH2", "luP2", "spkH", "spkP", "rH", "rP"};
  for (const char* a : split_arrays)
    if (!strcmp(what, a)) s.spike = true;  // the split forms are built on request
  std::string err;
  if (!opf::build_setup(&s, &err)) return fail(OPF_EINVAL, "opf_setup_query: " + err);
  const std::vector<double>* v = nullptr;
  std::vector<double> hop(s.hop.begin(), s.hop.end());
  if (!strcmp(what, "r")) v = &s.r;
  else if (!strcmp(what, "wq")) v = &s.wq;
  else if (!strcmp(what, "d1")) v = &s.d1;
  else if (!strcmp(what, "d2")) v = &s.d2;
  else if (!strcmp(what, "G")) v = &s.G;
  else if (!strcmp(what, "basis")) v = &s.basis;
  else if (!strcmp(what, "luH")) v = &s.luH;
  else if (!strcmp(what, "luP")) v = &s.luP;
  else if (!strcmp(what, "hop")) v = &hop;
  else if (!strcmp(what, "ainv")) v = &s.ainv;
  else if (!strcmp(what, "luH2")) v = &s.luH2;
  else if (!strcmp(what, "luP2")) v = &s.luP2;
  else if (!strcmp(what, "spkH")) v = &s.spkH;
  else if (!strcmp(what, "spkP")) v = &s.spkP;
  else if (!strcmp(what, "rH")) v = &s.rH;
  else if (!strcmp(what, "rP")) v = &s.rP;
  else return fail(OPF_EINVAL, std::string("opf_setup_query: unknown array ") + what);
  *len = (long)v->size();
  if (!out) return OPF_OK;
  if (cap < *len) return fail(OPF_EINVAL, "opf_setup_query: output too small");
  std::memcpy(out, v->data(), v->size() * sizeof(double));
  return OPF_OK;
}

}  // extern "C"

// ====================================================================== Newton-Krylov front end
namespace {

// Independent real coefficients of a state (state layout [3][M][nk][N]):
// m >= 1 all k (re, im); m = 0: k > 0 (re, im) and k = 0 (re only).
struct NkPack {
  int N, K, M, nk;
  long ndof;
  NkPack(int N_, int K_, int M_) : N(N_), K(K_), M(M_), nk(2 * K_ - 1) {
    ndof = 3L * N * ((long)(M - 1) * nk * 2 + (K - 1) * 2 + 1);
  }
  void pack(const double* st, double* x) const {  // st: interleaved complex
    long o = 0;
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < M; ++m)
        for (int kk = 0; kk < nk; ++kk) {
          const int k = kk - (K - 1);
          if (m == 0 && k < 0) continue;
          for (int n = 0; n < N; ++n) {
            const double* z = st + 2 * ((((long)c * M + m) * nk + kk) * N + n);
            x[o++] = z[0];
            if (!(m == 0 && k == 0)) x[o++] = z[1];
          }
        }
  }
  void unpack(const double* x, double* st) const {
    long o = 0;
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < M; ++m)
        for (int kk = 0; kk < nk; ++kk) {
          const int k = kk - (K - 1);
          if (m == 0 && k < 0) continue;
          for (int n = 0; n < N; ++n) {
            double* z = st + 2 * ((((long)c * M + m) * nk + kk) * N + n);
            z[0] = x[o++];
            z[1] = (m == 0 && k == 0) ? 0.0 : x[o++];
            if (m == 0 && k > 0) {  // conjugate partner
              double* w = st + 2 * ((((long)c * M + m) * nk + (nk - 1 - kk)) * N + n);
              w[0] = z[0];
              w[1] = -z[1];
            }
          }
        }
  }
};

struct NkCtx {
  Group g;
  Runner run;
  int N, K, M, m_p;
  double alpha;
  int count, nsteps;
  long ndof, n;  // n = ndof + free (T, s)
  opf_nk_opts o;
  std::vector<double> T, s;           // per problem: period, shift of the base point
  std::vector<std::vector<double>> phi, dphi_dt, dphi_ds, du_dt, du_dz, ubase;  // packed, base data
  std::vector<double> st;             // scratch state (interleaved complex, one trajectory)
  double2* forcing = nullptr;         // device copy of the body force (internal layout)
  NkPack pk;
  NkCtx(int N_, int K_, int M_) : pk(N_, K_, M_) {}
  ~NkCtx() {
    if (forcing) cudaFree(forcing);
  }
};

// The options' body force and frame rotation on the problems' group (shared
// by every trajectory of it, as on a handle).
int nk_apply_physics(NkCtx* c, const opf_nk_opts* o) {
  opf::Dims& d = c->g.d;
  const double x = o->rot[0], y = o->rot[1], z = o->rot[2];
  if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z))
    return fail(OPF_EINVAL, "nk: rotation must be finite");
  if ((x != 0.0 || y != 0.0) && c->m_p != 1)
    return fail(OPF_EINVAL, "nk: rotation about a transverse axis needs m_p = 1");
  d.rot_x = x;
  d.rot_y = y;
  d.rot_z = z;
  d.rotate = (x != 0.0 || y != 0.0 || z != 0.0) ? 1 : 0;
  if (o->forcing) {
    const size_t bytes = 3 * (size_t)d.F * sizeof(double2);
    CU(cudaMalloc((void**)&c->forcing, bytes));
    double2* abi = c->g.at(c->g.abi, 0);  // staging in the ABI layout
    CU(cudaMemcpyAsync(abi, o->forcing, bytes, cudaMemcpyHostToDevice, c->run.stream));
    opf::launch_abi_to_internal(c->g.single(0), abi, c->forcing, c->run.stream);
    CU(cudaStreamSynchronize(c->run.stream));
    CU(cudaGetLastError());
    d.forcing = c->forcing;
  }
  return OPF_OK;
}

// multiply each axial mode k of a state by e^{i alpha k s} (shift by s) and,
// if dz, by i alpha k (axial derivative)
void shift_state(const NkCtx& c, double* st, double s, bool dz) {
  const int nk = 2 * c.K - 1;
  for (int f = 0; f < 3; ++f)
    for (int m = 0; m < c.M; ++m)
      for (int kk = 0; kk < nk; ++kk) {
        const double ak = c.alpha * (kk - (c.K - 1));
        const double cr = std::cos(ak * s), ci = std::sin(ak * s);
        for (int n = 0; n < c.N; ++n) {
          double* z = &st[2 * ((((long)f * c.M + m) * nk + kk) * c.N + n)];
          double re = z[0] * cr - z[1] * ci, im = z[0] * ci + z[1] * cr;
          if (dz) {
            const double r2 = -ak * im, i2 = ak * re;
            re = r2;
            im = i2;
          }
          z[0] = re;
          z[1] = im;
        }
      }
}

// dt per problem from its period; operators refactored when any changed
int nk_set_periods(NkCtx* c, const int* idx, int cnt, const double* Ts) {
  bool changed = false;
  for (int j = 0; j < cnt; ++j) {
    const double dt = Ts[j] / c->nsteps;
    if (dt != c->g.dt[idx[j]]) {
      c->g.dt[idx[j]] = dt;
      changed = true;
    }
  }
  if (changed) return group_fill_setups(&c->g, false);
  return OPF_OK;
}

// integrate the given states (problem idx[j] uses trajectory idx[j]) for `steps`
// steps; states in/out as interleaved complex host arrays
int nk_integrate(NkCtx* c, int cnt, const int* idx, std::vector<std::vector<double>>& states, int steps) {
  for (int j = 0; j < cnt; ++j) {
    int rc = traj_set_state_host(&c->g, idx[j], states[j].data(), c->run.stream, false);
    if (rc) return rc;
  }
  int rc = runner_step(&c->run, steps);
  if (rc) return rc;
  for (int j = 0; j < cnt; ++j) {
    rc = traj_get_state(&c->g, idx[j], states[j].data(), true, c->run.stream);
    if (rc) return rc;
  }
  return OPF_OK;
}

long nk_state_len(const NkCtx* c) { return 2L * 3 * c->M * (2 * c->K - 1) * c->N; }

int nk_residual(void* vctx, int cnt, const int* idx, double* const* x, double* const* f, int commit) {
  NkCtx* c = (NkCtx*)vctx;
  const long L = nk_state_len(c);
  std::vector<std::vector<double>> u(cnt, std::vector<double>(L));
  std::vector<double> Ts(cnt), ss(cnt);
  for (int j = 0; j < cnt; ++j) {
    c->pk.unpack(x[j], u[j].data());
    long o = c->ndof;
    Ts[j] = c->o.fix_T ? c->T[idx[j]] : x[j][o++];
    ss[j] = c->o.fix_s ? c->s[idx[j]] : x[j][o++];
    if (!(Ts[j] > 0)) return fail(OPF_EINVAL, "nk: non-positive period");
  }
  int rc = nk_set_periods(c, idx, cnt, Ts.data());
  if (rc) return rc;
  std::vector<std::vector<double>> v = u;
  rc = nk_integrate(c, cnt, idx, v, c->nsteps);
  if (rc) return rc;
  for (int j = 0; j < cnt; ++j) {
    std::vector<double> w = v[j];
    shift_state(*c, w.data(), ss[j], false);
    c->pk.pack(w.data(), f[j]);
    for (long t = 0; t < c->ndof; ++t) f[j][t] -= x[j][t];
    for (long t = c->ndof; t < c->n; ++t) f[j][t] = 0.0;
  }
  if (!commit) return OPF_OK;
  // base data for the Jacobian-vector products at these points
  std::vector<std::vector<double>> v1 = v, u1 = u;
  rc = nk_integrate(c, cnt, idx, v1, 1);  // one more step from Phi_T(u)
  if (rc) return rc;
  rc = nk_integrate(c, cnt, idx, u1, 1);  // one step from u
  if (rc) return rc;
  for (int j = 0; j < cnt; ++j) {
    const int i = idx[j];
    const double dt = c->g.dt[i];
    c->T[i] = Ts[j];
    c->s[i] = ss[j];
    std::vector<double> w = v[j];
    shift_state(*c, w.data(), ss[j], false);
    c->phi[i].resize(c->ndof);
    c->pk.pack(w.data(), c->phi[i].data());
    std::vector<double> a = v1[j];
    for (long t = 0; t < L; ++t) a[t] = (a[t] - v[j][t]) / dt;
    shift_state(*c, a.data(), ss[j], false);
    c->dphi_dt[i].resize(c->ndof);
    c->pk.pack(a.data(), c->dphi_dt[i].data());
    std::vector<double> b = v[j];
    shift_state(*c, b.data(), ss[j], true);
    c->dphi_ds[i].resize(c->ndof);
    c->pk.pack(b.data(), c->dphi_ds[i].data());
    std::vector<double> e = u1[j];
    for (long t = 0; t < L; ++t) e[t] = (e[t] - u[j][t]) / dt;
    c->du_dt[i].resize(c->ndof);
    c->pk.pack(e.data(), c->du_dt[i].data());
    std::vector<double> zz = u[j];
    shift_state(*c, zz.data(), 0.0, true);
    c->du_dz[i].resize(c->ndof);
    c->pk.pack(zz.data(), c->du_dz[i].data());
    c->ubase[i].assign(x[j], x[j] + c->ndof);
  }
  return OPF_OK;
}

int nk_jv(void* vctx, int cnt, const int* idx, double* const* x, double* const* v, double* const* jv) {
  NkCtx* c = (NkCtx*)vctx;
  const long L = nk_state_len(c);
  {  // a rejected trial may have left its period in the setup: back to the base point's
    std::vector<double> Tb(cnt);
    for (int j = 0; j < cnt; ++j) Tb[j] = c->T[idx[j]];
    int rc0 = nk_set_periods(c, idx, cnt, Tb.data());
    if (rc0) return rc0;
  }
  std::vector<std::vector<double>> up(cnt, std::vector<double>(L));
  std::vector<double> eps(cnt);
  std::vector<double> tmp(c->ndof);
  for (int j = 0; j < cnt; ++j) {
    double xn = 0.0, vn = 0.0;
    for (long t = 0; t < c->ndof; ++t) {
      xn += x[j][t] * x[j][t];
      vn += v[j][t] * v[j][t];
    }
    eps[j] = vn > 0 ? c->o.eps * std::sqrt(xn / vn) : 1.0;
    for (long t = 0; t < c->ndof; ++t) tmp[t] = x[j][t] + eps[j] * v[j][t];
    c->pk.unpack(tmp.data(), up[j].data());
  }
  int rc = nk_integrate(c, cnt, idx, up, c->nsteps);
  if (rc) return rc;
  for (int j = 0; j < cnt; ++j) {
    const int i = idx[j];
    shift_state(*c, up[j].data(), c->s[i], false);
    c->pk.pack(up[j].data(), jv[j]);
    const double dT = c->o.fix_T ? 0.0 : v[j][c->ndof];
    const double ds = c->o.fix_s ? 0.0 : v[j][c->ndof + (c->o.fix_T ? 0 : 1)];
    double pt = 0.0, pz = 0.0;
    for (long t = 0; t < c->ndof; ++t) {
      jv[j][t] = (jv[j][t] - c->phi[i][t]) / eps[j] - v[j][t] + dT * c->dphi_dt[i][t] + ds * c->dphi_ds[i][t];
      pt += c->du_dt[i][t] * v[j][t];
      pz += c->du_dz[i][t] * v[j][t];
    }
    long o = c->ndof;
    if (!c->o.fix_T) jv[j][o++] = pt;
    if (!c->o.fix_s) jv[j][o++] = pz;
  }
  return OPF_OK;
}

}  // namespace

extern "C" int opf_nk_solve(int N, int K, int M, int m_p, double alpha, double Re, int count,
                            double* states, double* T, double* s, const opf_nk_opts* o,
                            double* residual, int* iters) {
  if (count < 1 || !states || !T || !s || !o || !(o->dt > 0) || !(o->eps > 0))
    return fail(OPF_EINVAL, "opf_nk_solve: bad arguments");
  NkCtx* c = new NkCtx(N, K, M);
  c->N = N;
  c->K = K;
  c->M = M;
  c->m_p = m_p;
  c->alpha = alpha;
  c->count = count;
  c->o = *o;
  double Tmax = 0.0;
  for (int i = 0; i < count; ++i) Tmax = std::max(Tmax, T[i]);
  c->nsteps = std::max(1, (int)std::ceil(Tmax / o->dt - 1e-9));
  std::vector<double> Re_v(count, Re), dt_v(count);
  for (int i = 0; i < count; ++i) dt_v[i] = T[i] / c->nsteps;
  // periods may diverge during the solve: every problem gets its own setup
  int rc = group_build(&c->g, N, K, M, m_p, alpha, count, Re_v.data(), dt_v.data(), true);
  if (rc == OPF_OK) rc = runner_init(&c->run);
  if (rc == OPF_OK) rc = nk_apply_physics(c, o);
  if (rc != OPF_OK) {
    group_free(&c->g);
    runner_free(&c->run);
    delete c;
    return rc;
  }
  c->run.groups = {&c->g};
  c->run.precision = o->precision;
  c->ndof = c->pk.ndof;
  c->n = c->ndof + (o->fix_T ? 0 : 1) + (o->fix_s ? 0 : 1);
  c->T.assign(T, T + count);
  c->s.assign(s, s + count);
  c->phi.resize(count);
  c->dphi_dt.resize(count);
  c->dphi_ds.resize(count);
  c->du_dt.resize(count);
  c->du_dz.resize(count);
  c->ubase.resize(count);
  const long L = nk_state_len(c);
  std::vector<double> x((size_t)count * c->n), scale(count);
  for (int i = 0; i < count; ++i) {
    double* xi = &x[(size_t)i * c->n];
    c->pk.pack(states + (size_t)i * L, xi);
    long q = c->ndof;
    if (!o->fix_T) xi[q++] = T[i];
    if (!o->fix_s) xi[q++] = s[i];
    double nn = 0.0;
    for (long t = 0; t < c->ndof; ++t) nn += xi[t] * xi[t];
    scale[i] = std::sqrt(nn);
  }
  std::vector<double> res(count, 0.0);
  std::vector<int> it(count, 0);
  rc = opf_nk_core((int)c->n, count, x.data(), scale.data(), nk_residual, nk_jv, c, o, res.data(), it.data());
  if (rc == OPF_OK) {
    for (int i = 0; i < count; ++i) {
      const double* xi = &x[(size_t)i * c->n];
      c->pk.unpack(xi, states + (size_t)i * L);
      long q = c->ndof;
      if (!o->fix_T) T[i] = xi[q++];
      if (!o->fix_s) s[i] = xi[q++];
      if (residual) residual[i] = res[i];
      if (iters) iters[i] = it[i];
    }
  }
  runner_free(&c->run);
  group_free(&c->g);
  delete c;
  return rc;
}

// ---- multiple shooting (section 2: the orbit is split into S sections, each
// integrated over T/S as its own trajectory of the batched group).  Unknowns
// per problem: the S section starts (u_0 .. u_{S-1}), then T and s unless
// fixed.  Residual: F_q = Phi_{T/S}(u_q) - u_{q+1} (q < S-1),
// F_{S-1} = sigma_s Phi_{T/S}(u_{S-1}) - u_0; phase conditions on section 0.
// Problem i's section q is trajectory i*S + q.
namespace {
struct MsCtx {
  NkCtx* c;
  int S;
  // per trajectory (i*S + q): packed base point, Phi(u_q) (the last one shifted),
  // d/dt of it; per problem: d/ds of the shifted last section, du_0/dt, du_0/dz
  std::vector<std::vector<double>> ubase, phi, dphi_dt, dphi_ds, du_dt, du_dz;
};

int ms_set_periods(MsCtx* m, const int* idx, int cnt, const double* Ts) {
  NkCtx* c = m->c;
  bool changed = false;
  for (int j = 0; j < cnt; ++j)
    for (int q = 0; q < m->S; ++q) {
      const int t = idx[j] * m->S + q;
      const double dt = Ts[j] / (m->S * c->nsteps);
      if (dt != c->g.dt[t]) {
        c->g.dt[t] = dt;
        changed = true;
      }
    }
  if (changed) return group_fill_setups(&c->g, false);
  return OPF_OK;
}

int ms_residual(void* vctx, int cnt, const int* idx, double* const* x, double* const* f, int commit) {
  MsCtx* m = (MsCtx*)vctx;
  NkCtx* c = m->c;
  const int S = m->S;
  const long L = nk_state_len(c), nd = c->ndof;
  std::vector<int> tr(cnt * S);
  std::vector<std::vector<double>> u(cnt * S, std::vector<double>(L));
  std::vector<double> Ts(cnt), ss(cnt);
  for (int j = 0; j < cnt; ++j) {
    long o = S * nd;
    Ts[j] = c->o.fix_T ? c->T[idx[j]] : x[j][o++];
    ss[j] = c->o.fix_s ? c->s[idx[j]] : x[j][o++];
    if (!(Ts[j] > 0)) return fail(OPF_EINVAL, "nk: non-positive period");
    for (int q = 0; q < S; ++q) {
      tr[j * S + q] = idx[j] * S + q;
      c->pk.unpack(x[j] + q * nd, u[j * S + q].data());
    }
  }
  int rc = ms_set_periods(m, idx, cnt, Ts.data());
  if (rc) return rc;
  std::vector<std::vector<double>> v = u;
  rc = nk_integrate(c, cnt * S, tr.data(), v, c->nsteps);
  if (rc) return rc;
  std::vector<double> w(L), pk(nd);
  for (int j = 0; j < cnt; ++j) {
    for (int q = 0; q < S; ++q) {
      w = v[j * S + q];
      if (q == S - 1) shift_state(*c, w.data(), ss[j], false);
      c->pk.pack(w.data(), pk.data());
      const double* next = x[j] + ((q + 1) % S) * nd;
      for (long t = 0; t < nd; ++t) f[j][q * nd + t] = pk[t] - next[t];
    }
    for (long t = S * nd; t < c->n; ++t) f[j][t] = 0.0;
  }
  if (!commit) return OPF_OK;
  std::vector<std::vector<double>> v1 = v, u1 = u;
  rc = nk_integrate(c, cnt * S, tr.data(), v1, 1);  // one more step from each Phi(u_q)
  if (rc) return rc;
  rc = nk_integrate(c, cnt * S, tr.data(), u1, 1);  // one step from each u_q
  if (rc) return rc;
  for (int j = 0; j < cnt; ++j) {
    const int i = idx[j];
    c->T[i] = Ts[j];
    c->s[i] = ss[j];
    for (int q = 0; q < S; ++q) {
      const int t = i * S + q, k = j * S + q;
      const double dt = c->g.dt[t];
      const bool last = q == S - 1;
      w = v[k];
      if (last) shift_state(*c, w.data(), ss[j], false);
      m->phi[t].resize(nd);
      c->pk.pack(w.data(), m->phi[t].data());
      std::vector<double> a = v1[k];
      for (long e = 0; e < L; ++e) a[e] = (a[e] - v[k][e]) / dt;
      if (last) shift_state(*c, a.data(), ss[j], false);
      m->dphi_dt[t].resize(nd);
      c->pk.pack(a.data(), m->dphi_dt[t].data());
      m->ubase[t].assign(x[j] + q * nd, x[j] + (q + 1) * nd);
      if (last) {
        std::vector<double> b = v[k];
        shift_state(*c, b.data(), ss[j], true);
        m->dphi_ds[i].resize(nd);
        c->pk.pack(b.data(), m->dphi_ds[i].data());
      }
      if (q == 0) {
        std::vector<double> e1 = u1[k];
        for (long e = 0; e < L; ++e) e1[e] = (e1[e] - u[k][e]) / dt;
        m->du_dt[i].resize(nd);
        c->pk.pack(e1.data(), m->du_dt[i].data());
        std::vector<double> zz = u[k];
        shift_state(*c, zz.data(), 0.0, true);
        m->du_dz[i].resize(nd);
        c->pk.pack(zz.data(), m->du_dz[i].data());
      }
    }
  }
  return OPF_OK;
}

int ms_jv(void* vctx, int cnt, const int* idx, double* const* /*x: the base points, held in the context*/,
          double* const* v, double* const* jv) {
  MsCtx* m = (MsCtx*)vctx;
  NkCtx* c = m->c;
  const int S = m->S;
  const long L = nk_state_len(c), nd = c->ndof;
  {  // a rejected trial may have left its period in the setup: back to the base point's
    std::vector<double> Tb(cnt);
    for (int j = 0; j < cnt; ++j) Tb[j] = c->T[idx[j]];
    int rc0 = ms_set_periods(m, idx, cnt, Tb.data());
    if (rc0) return rc0;
  }
  std::vector<int> tr(cnt * S);
  std::vector<std::vector<double>> up(cnt * S, std::vector<double>(L));
  std::vector<double> eps(cnt * S), tmp(nd);
  for (int j = 0; j < cnt; ++j)
    for (int q = 0; q < S; ++q) {
      const int t = idx[j] * S + q;
      tr[j * S + q] = t;
      const std::vector<double>& ub = m->ubase[t];
      const double* d = v[j] + q * nd;
      double un = 0.0, vn = 0.0;
      for (long e = 0; e < nd; ++e) {
        un += ub[e] * ub[e];
        vn += d[e] * d[e];
      }
      const double ep = vn > 0 ? c->o.eps * std::sqrt(un / vn) : 1.0;
      eps[j * S + q] = ep;
      for (long e = 0; e < nd; ++e) tmp[e] = ub[e] + ep * d[e];
      c->pk.unpack(tmp.data(), up[j * S + q].data());
    }
  int rc = nk_integrate(c, cnt * S, tr.data(), up, c->nsteps);
  if (rc) return rc;
  std::vector<double> pk(nd);
  for (int j = 0; j < cnt; ++j) {
    const int i = idx[j];
    const double dT = c->o.fix_T ? 0.0 : v[j][S * nd];
    const double ds = c->o.fix_s ? 0.0 : v[j][S * nd + (c->o.fix_T ? 0 : 1)];
    for (int q = 0; q < S; ++q) {
      const int t = i * S + q, k = j * S + q;
      if (q == S - 1) shift_state(*c, up[k].data(), c->s[i], false);
      c->pk.pack(up[k].data(), pk.data());
      const double* dn = v[j] + ((q + 1) % S) * nd;
      for (long e = 0; e < nd; ++e) {
        double r = (pk[e] - m->phi[t][e]) / eps[k] - dn[e] + (dT / S) * m->dphi_dt[t][e];
        if (q == S - 1) r += ds * m->dphi_ds[i][e];
        jv[j][q * nd + e] = r;
      }
    }
    double pt = 0.0, pz = 0.0;
    for (long e = 0; e < nd; ++e) {
      pt += m->du_dt[i][e] * v[j][e];
      pz += m->du_dz[i][e] * v[j][e];
    }
    long o = S * nd;
    if (!c->o.fix_T) jv[j][o++] = pt;
    if (!c->o.fix_s) jv[j][o++] = pz;
  }
  return OPF_OK;
}
}  // namespace

extern "C" int opf_nk_solve_ms(int N, int K, int M, int m_p, double alpha, double Re, int count, int S,
                               double* states, double* T, double* s, const opf_nk_opts* o, double* residual,
                               int* iters) {
  if (count < 1 || S < 1 || !states || !T || !s || !o || !(o->dt > 0) || !(o->eps > 0))
    return fail(OPF_EINVAL, "opf_nk_solve_ms: bad arguments");
  for (int i = 0; i < count; ++i)
    if (!(T[i] > 0)) return fail(OPF_EINVAL, "opf_nk_solve_ms: periods must be positive");
  NkCtx* c = new NkCtx(N, K, M);
  c->N = N;
  c->K = K;
  c->M = M;
  c->m_p = m_p;
  c->alpha = alpha;
  c->count = count;
  c->o = *o;
  double Tmax = 0.0;
  for (int i = 0; i < count; ++i) Tmax = std::max(Tmax, T[i]);
  c->nsteps = std::max(1, (int)std::ceil(Tmax / S / o->dt - 1e-9));  // steps per section
  const int ntr = count * S;
  std::vector<double> Re_v(ntr, Re), dt_v(ntr);
  for (int t = 0; t < ntr; ++t) dt_v[t] = T[t / S] / (S * c->nsteps);
  int rc = group_build(&c->g, N, K, M, m_p, alpha, ntr, Re_v.data(), dt_v.data(), true);
  if (rc == OPF_OK) rc = runner_init(&c->run);
  if (rc == OPF_OK) rc = nk_apply_physics(c, o);
  if (rc != OPF_OK) {
    group_free(&c->g);
    runner_free(&c->run);
    delete c;
    return rc;
  }
  c->run.groups = {&c->g};
  c->run.precision = o->precision;
  c->ndof = c->pk.ndof;
  c->n = S * c->ndof + (o->fix_T ? 0 : 1) + (o->fix_s ? 0 : 1);
  c->T.assign(T, T + count);
  c->s.assign(s, s + count);
  MsCtx m{c, S, {}, {}, {}, {}, {}, {}};
  m.ubase.resize(ntr);
  m.phi.resize(ntr);
  m.dphi_dt.resize(ntr);
  m.dphi_ds.resize(count);
  m.du_dt.resize(count);
  m.du_dz.resize(count);
  const long L = nk_state_len(c);
  std::vector<double> x((size_t)count * c->n), scale(count);
  for (int i = 0; i < count; ++i) {
    double* xi = &x[(size_t)i * c->n];
    for (int q = 0; q < S; ++q) c->pk.pack(states + ((size_t)i * S + q) * L, xi + q * c->ndof);
    long q = S * c->ndof;
    if (!o->fix_T) xi[q++] = T[i];
    if (!o->fix_s) xi[q++] = s[i];
    double nn = 0.0;
    for (long t = 0; t < S * c->ndof; ++t) nn += xi[t] * xi[t];
    scale[i] = std::sqrt(nn);
  }
  std::vector<double> res(count, 0.0);
  std::vector<int> it(count, 0);
  rc = opf_nk_core((int)c->n, count, x.data(), scale.data(), ms_residual, ms_jv, &m, o, res.data(), it.data());
  if (rc == OPF_OK) {
    for (int i = 0; i < count; ++i) {
      const double* xi = &x[(size_t)i * c->n];
      for (int q = 0; q < S; ++q) c->pk.unpack(xi + q * c->ndof, states + ((size_t)i * S + q) * L);
      long q = S * c->ndof;
      if (!o->fix_T) T[i] = xi[q++];
      if (!o->fix_s) s[i] = xi[q++];
      if (residual) residual[i] = res[i];
      if (iters) iters[i] = it[i];
    }
  }
  runner_free(&c->run);
  group_free(&c->g);
  delete c;
  return rc;
}

// ---- Floquet multipliers / eigenvalues of invariant solutions
namespace {
struct FqCtx {
  NkCtx* c;
  double eps;
  std::vector<std::vector<double>> base;  // packed sigma_s Phi_T(u) per problem
};

// av = (sigma_s Phi_T(u + e v) - sigma_s Phi_T(u)) / e, e = eps |u| / |v|
int fq_apply(void* vctx, int cnt, const int* idx, double* const* v, double* const* av) {
  FqCtx* f = (FqCtx*)vctx;
  NkCtx* c = f->c;
  const long L = nk_state_len(c);
  std::vector<std::vector<double>> up(cnt, std::vector<double>(L));
  std::vector<double> e(cnt), tmp(c->ndof);
  for (int j = 0; j < cnt; ++j) {
    const std::vector<double>& u = c->ubase[idx[j]];
    double un = 0.0, vn = 0.0;
    for (long t = 0; t < c->ndof; ++t) {
      un += u[t] * u[t];
      vn += v[j][t] * v[j][t];
    }
    e[j] = vn > 0 ? f->eps * std::sqrt(un / vn) : 1.0;
    for (long t = 0; t < c->ndof; ++t) tmp[t] = u[t] + e[j] * v[j][t];
    c->pk.unpack(tmp.data(), up[j].data());
  }
  int rc = nk_integrate(c, cnt, idx, up, c->nsteps);
  if (rc) return rc;
  for (int j = 0; j < cnt; ++j) {
    const int i = idx[j];
    shift_state(*c, up[j].data(), c->s[i], false);
    c->pk.pack(up[j].data(), av[j]);
    for (long t = 0; t < c->ndof; ++t) av[j][t] = (av[j][t] - f->base[i][t]) / e[j];
  }
  return OPF_OK;
}
}  // namespace

extern "C" int opf_floquet(int N, int K, int M, int m_p, double alpha, double Re, int count, const double* states,
                           const double* T, const double* s, int kdim, int nev, double dt, double eps,
                           int precision, unsigned long long seed, const double* start, double* eig_re,
                           double* eig_im, double* resid) {
  if (count < 1 || !states || !T || !s || kdim < 1 || nev < 1 || nev > kdim || !(dt > 0) || !(eps > 0) ||
      !eig_re || !eig_im || (precision != 0 && precision != 1))
    return fail(OPF_EINVAL, "opf_floquet: bad arguments");
  for (int i = 0; i < count; ++i)
    if (!(T[i] > 0)) return fail(OPF_EINVAL, "opf_floquet: periods must be positive");
  NkCtx* c = new NkCtx(N, K, M);
  c->N = N;
  c->K = K;
  c->M = M;
  c->m_p = m_p;
  c->alpha = alpha;
  c->count = count;
  double Tmax = 0.0;
  for (int i = 0; i < count; ++i) Tmax = std::max(Tmax, T[i]);
  c->nsteps = std::max(1, (int)std::ceil(Tmax / dt - 1e-9));
  std::vector<double> Re_v(count, Re), dt_v(count);
  for (int i = 0; i < count; ++i) dt_v[i] = T[i] / c->nsteps;
  int rc = group_build(&c->g, N, K, M, m_p, alpha, count, Re_v.data(), dt_v.data(), true);
  if (rc == OPF_OK) rc = runner_init(&c->run);
  if (rc != OPF_OK) {
    group_free(&c->g);
    runner_free(&c->run);
    delete c;
    return rc;
  }
  c->run.groups = {&c->g};
  c->run.precision = precision;
  c->ndof = c->pk.ndof;
  c->n = c->ndof;
  c->T.assign(T, T + count);
  c->s.assign(s, s + count);
  c->ubase.resize(count);
  FqCtx f{c, eps, {}};
  f.base.resize(count);
  const long L = nk_state_len(c);
  std::vector<int> all(count);
  std::vector<std::vector<double>> u(count);
  for (int i = 0; i < count; ++i) {
    all[i] = i;
    c->ubase[i].resize(c->ndof);
    c->pk.pack(states + (size_t)i * L, c->ubase[i].data());
    u[i].assign(states + (size_t)i * L, states + (size_t)(i + 1) * L);
  }
  rc = nk_integrate(c, count, all.data(), u, c->nsteps);
  if (rc == OPF_OK) {
    // base points, and seeded starting vectors (SplitMix64 uniforms in [-1, 1))
    std::vector<double> v0((size_t)count * c->ndof);
    unsigned long long z = seed;
    for (size_t t = 0; t < v0.size(); ++t) {
      z += 0x9E3779B97F4A7C15ull;
      unsigned long long q = z;
      q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ull;
      q = (q ^ (q >> 27)) * 0x94D049BB133111EBull;
      q ^= q >> 31;
      v0[t] = 2.0 * ((double)(q >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
    if (start)  // caller's starting vectors, state layout
      for (int i = 0; i < count; ++i) c->pk.pack(start + (size_t)i * L, &v0[(size_t)i * c->ndof]);
    for (int i = 0; i < count; ++i) {
      shift_state(*c, u[i].data(), c->s[i], false);
      f.base[i].resize(c->ndof);
      c->pk.pack(u[i].data(), f.base[i].data());
    }
    rc = opf_arnoldi_core((int)c->ndof, count, v0.data(), kdim, nev, fq_apply, &f, eig_re, eig_im, resid, nullptr);
  }
  runner_free(&c->run);
  group_free(&c->g);
  delete c;
  return rc;
}
