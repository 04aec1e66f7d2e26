// C ABI of libopf (declared in include/opf.h): handle life cycle, state
// transfer, and the predictor-corrector orchestration of section 2.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
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
constexpr int kMaxSlots = 32;
const char* kNames[] = {"curl", "zsynth", "product", "zanalysis", "solve"};
constexpr int kNumNames = 5;
}  // namespace

struct opf_ctx {
  opf::Setup hs;
  opf::DevSetup ds;
  opf::Dims d{};
  opf::FftPlan pz{}, pth{};
  double2 *U = nullptr, *U1 = nullptr, *Nj = nullptr, *Nq = nullptr, *W6 = nullptr;
  double2 *Z6 = nullptr, *ZN = nullptr, *abi = nullptr, *tmpU = nullptr;
  float2 *W6f = nullptr, *Z6f = nullptr, *ZNf = nullptr;  // mixed-precision intermediates
  double2* Nlin = nullptr;                                // FP64 linear terms (mixed)
  double *beta_p = nullptr, *partial = nullptr, *out3 = nullptr, *out2 = nullptr;
  int* flag = nullptr;
  int nblk_energy = 0;
  cudaStream_t own = nullptr, stream = nullptr;
  int precision = 0, n_corr = 1, use_graph = 1, timing = 0;
  cudaGraphExec_t gexec = nullptr;
  double time = 0.0;
  int device = 0;
  std::vector<void*> allocs;
  // per-launch timing
  cudaEvent_t ev[kMaxSlots][2];
  int slot_name[kMaxSlots];
  int nslots = 0, graph_nslots = 0;
  bool events_made = false;
  double tot_ms[kNumNames] = {0};
  int tot_n[kNumNames] = {0};
};

namespace {

template <typename P>
int dalloc(opf_ctx* h, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return fail(OPF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(q);
  *p = (P*)q;
  return OPF_OK;
}

template <typename T>
int upload(opf_ctx* h, T** dst, const std::vector<T>& v) {
  int rc = dalloc(h, dst, v.size() * sizeof(T) + 16);
  if (rc) return rc;
  CU(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return OPF_OK;
}

int upload_setup(opf_ctx* h) {
  const opf::Setup& s = h->hs;
  int rc;
  if ((rc = upload(h, &h->ds.rinv, s.rinv))) return rc;
  if ((rc = upload(h, &h->ds.d1, s.d1))) return rc;
  if ((rc = upload(h, &h->ds.wq, s.wq))) return rc;
  if ((rc = upload(h, &h->ds.hop, s.hop))) return rc;
  if ((rc = upload(h, &h->ds.luH, s.luH))) return rc;
  if ((rc = upload(h, &h->ds.luP, s.luP))) return rc;
  if ((rc = upload(h, &h->ds.basis, s.basis))) return rc;
  double* ai = nullptr;
  if ((rc = upload(h, &ai, s.ainv))) return rc;
  h->ds.ainv = (double2*)ai;
  if ((rc = upload(h, &h->ds.G, s.G))) return rc;
  auto twiddles = [&](int n, double2** out, float2** out32) -> int {
    std::vector<double2> t(n);
    std::vector<float2> t32(n);
    for (int i = 0; i < n; ++i) {
      const long double a = 2.0L * 3.14159265358979323846264338327950288L * i / n;
      t[i] = double2{(double)cosl(a), (double)sinl(a)};
      t32[i] = float2{(float)t[i].x, (float)t[i].y};
    }
    int r2 = upload(h, out, t);
    if (r2) return r2;
    return upload(h, out32, t32);
  };
  if ((rc = twiddles(h->d.nz, &h->ds.tw_z, &h->ds.tw_z32))) return rc;
  if ((rc = twiddles(h->d.nth, &h->ds.tw_th, &h->ds.tw_th32))) return rc;
  return OPF_OK;
}

void free_all(opf_ctx* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->events_made)
    for (int i = 0; i < kMaxSlots; ++i) {
      cudaEventDestroy(h->ev[i][0]);
      cudaEventDestroy(h->ev[i][1]);
    }
  if (h->own) cudaStreamDestroy(h->own);
}

// ---- step orchestration
void begin(opf_ctx* h, int name) {
  if (!h->timing || h->nslots >= kMaxSlots) return;
  h->slot_name[h->nslots] = name;
  // external: inside stream capture this becomes an event-record node
  cudaEventRecordWithFlags(h->ev[h->nslots][0], h->stream, cudaEventRecordExternal);
}
void end(opf_ctx* h) {
  if (!h->timing || h->nslots >= kMaxSlots) return;
  cudaEventRecordWithFlags(h->ev[h->nslots][1], h->stream, cudaEventRecordExternal);
  ++h->nslots;
}

void enqueue_nonlinear(opf_ctx* h, const double2* U, double2* Nout) {
  const opf::Dims& d = h->d;
  if (h->precision == 1) {
    begin(h, 0);
    opf::launch_curl_split32(d, h->ds, U, h->W6f, h->Nlin, h->stream);
    end(h);
    begin(h, 1);
    opf::launch_zsynth32(d, h->ds, h->pz, h->W6f, h->Z6f, h->stream);
    end(h);
    begin(h, 2);
    opf::launch_product32(d, h->ds, h->pth, h->Z6f, h->ZNf, h->stream);
    end(h);
    begin(h, 3);
    opf::launch_zanalysis32(d, h->ds, h->pz, h->ZNf, h->Nlin, Nout, h->stream);
    end(h);
    return;
  }
  begin(h, 0);
  opf::launch_curl(d, h->ds, U, h->W6, h->stream);
  end(h);
  begin(h, 1);
  opf::launch_zsynth(d, h->ds, h->pz, h->W6, h->Z6, h->stream);
  end(h);
  begin(h, 2);
  opf::launch_product(d, h->ds, h->pth, h->Z6, h->ZN, h->stream);
  end(h);
  begin(h, 3);
  opf::launch_zanalysis(d, h->ds, h->pz, h->ZN, Nout, h->stream);
  end(h);
}

void enqueue_solve(opf_ctx* h, const double2* Na, const double2* Nb, double wa, double wb,
                   double2* Uout) {
  opf::SolveArgs a{h->U, Na, Nb, wa, wb, Uout, h->beta_p};
  begin(h, 4);
  opf::launch_solve(h->d, h->ds, a, h->hs.flux_G, h->hs.nJ, h->stream);
  end(h);
}

// One predictor-corrector step (section 2): predictor with N_j, then n_corr
// corrector passes with c N^q + (1 - c) N_j, each solved from u_j.
void enqueue_step(opf_ctx* h) {
  const double c = h->d.c;
  enqueue_nonlinear(h, h->U, h->Nj);
  enqueue_solve(h, h->Nj, nullptr, 1.0, 0.0, h->U1);
  for (int q = 0; q < h->n_corr; ++q) {
    enqueue_nonlinear(h, h->U1, h->Nq);
    enqueue_solve(h, h->Nq, h->Nj, c, 1.0 - c, q == h->n_corr - 1 ? h->U : h->U1);
  }
}

int harvest_timing(opf_ctx* h) {
  if (!h->timing) return OPF_OK;
  for (int i = 0; i < h->nslots; ++i) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, h->ev[i][0], h->ev[i][1]));
    h->tot_ms[h->slot_name[i]] += ms;
    h->tot_n[h->slot_name[i]] += 1;
  }
  return OPF_OK;
}

int check_handle(opf_t* h) { return h ? OPF_OK : fail(OPF_EINVAL, "NULL handle"); }

bool smooth235(int n) {
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

}  // namespace

extern "C" {

const char* opf_last_error(void) { return g_err.c_str(); }

opf_t* opf_create(int N, int K, int M, int m_p, double alpha, double Re, double dt) {
  if (N < 9 || K < 1 || M < 1 || m_p < 1 || !(alpha > 0) || !(Re > 0) || !(dt > 0)) {
    fail(OPF_EINVAL, "opf_create: need N>=9, K>=1, M>=1, m_p>=1, alpha>0, Re>0, dt>0");
    return nullptr;
  }
  if (!smooth235(3 * K) || !smooth235(3 * M)) {
    fail(OPF_EINVAL, "opf_create: 3K and 3M must have no prime factor other than 2, 3, 5");
    return nullptr;
  }
  opf_ctx* h = new opf_ctx();
  h->hs.N = N;
  h->hs.K = K;
  h->hs.M = M;
  h->hs.m_p = m_p;
  h->hs.alpha = alpha;
  h->hs.Re = Re;
  h->hs.dt = dt;
  h->hs.c = 0.5;
  std::string err;
  if (!opf::build_setup(&h->hs, &err)) {
    fail(OPF_EINVAL, "opf_create: " + err);
    delete h;
    return nullptr;
  }
  opf::Dims& d = h->d;
  d.N = N;
  d.K = K;
  d.M = M;
  d.m_p = m_p;
  d.nk = 2 * K - 1;
  d.nz = 3 * K;
  d.nth = 3 * M;
  d.alpha = alpha;
  d.Re = Re;
  d.dt = dt;
  d.c = 0.5;
  d.F = (long)M * N * d.nk;
  opf::choose_chunks(&d);
  if (!opf::make_plan(d.nz, &h->pz) || !opf::make_plan(d.nth, &h->pth)) {
    fail(OPF_EINVAL, "opf_create: no FFT plan for 3K or 3M");
    delete h;
    return nullptr;
  }
  auto bail = [&](int) -> opf_t* {
    std::string keep = g_err;
    free_all(h);
    delete h;
    g_err = keep;
    return nullptr;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    fail(OPF_ECUDA, "opf_create: no CUDA device");
    return bail(0);
  }
  const size_t F16 = (size_t)d.F * sizeof(double2);
  const size_t P16 = (size_t)N * d.nz * M * sizeof(double2);
  if (dalloc(h, &h->U, 3 * F16) || dalloc(h, &h->U1, 3 * F16) || dalloc(h, &h->Nj, 3 * F16) ||
      dalloc(h, &h->Nq, 3 * F16) || dalloc(h, &h->W6, 6 * F16) || dalloc(h, &h->Z6, 6 * P16) ||
      dalloc(h, &h->ZN, 3 * P16) || dalloc(h, &h->abi, 3 * F16) || dalloc(h, &h->tmpU, 3 * F16) ||
      dalloc(h, &h->beta_p, 16) || dalloc(h, &h->out3, 32) || dalloc(h, &h->out2, 16) ||
      dalloc(h, &h->flag, 16) || dalloc(h, &h->W6f, 6 * F16 / 2) || dalloc(h, &h->Z6f, 6 * P16 / 2) ||
      dalloc(h, &h->ZNf, 3 * P16 / 2) || dalloc(h, &h->Nlin, 3 * F16))
    return bail(0);
  h->nblk_energy = opf::energy_blocks(d);
  if (dalloc(h, &h->partial, (size_t)2 * h->nblk_energy * sizeof(double))) return bail(0);
  if (upload_setup(h)) return bail(0);
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) {
    fail(OPF_ECUDA, "opf_create: stream");
    return bail(0);
  }
  h->stream = h->own;
  if (!opf::prepare_kernel_attrs(d)) {
    fail(OPF_EINVAL, "opf_create: resolution needs more shared memory than a block has");
    return bail(0);
  }
  for (int i = 0; i < kMaxSlots; ++i) {
    cudaEventCreate(&h->ev[i][0]);
    cudaEventCreate(&h->ev[i][1]);
  }
  h->events_made = true;
  cudaMemset(h->U, 0, 3 * F16);
  cudaMemset(h->beta_p, 0, 16);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fail(OPF_ECUDA, std::string("opf_create: ") + cudaGetErrorString(e));
    return bail(0);
  }
  return h;
}

void opf_destroy(opf_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

int opf_set_state_device(opf_t* h, const double* d_coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!d_coeffs) return fail(OPF_EINVAL, "opf_set_state: NULL buffer");
  const size_t bytes = 3 * (size_t)h->d.F * sizeof(double2);
  CU(cudaMemcpyAsync(h->abi, d_coeffs, bytes, cudaMemcpyDeviceToDevice, h->stream));
  opf::launch_nan_check((const double*)h->abi, 6 * h->d.F, h->flag, h->stream);
  int flag = 0;
  CU(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (flag) return fail(OPF_ENAN, "opf_set_state: non-finite coefficient; state unchanged");
  opf::launch_abi_to_internal(h->d, h->abi, h->U, h->stream);
  CU(cudaMemsetAsync(h->beta_p, 0, sizeof(double), h->stream));
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  return OPF_OK;
}

int opf_set_state(opf_t* h, const double* coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!coeffs) return fail(OPF_EINVAL, "opf_set_state: NULL buffer");
  const size_t bytes = 3 * (size_t)h->d.F * sizeof(double2);
  CU(cudaMemcpyAsync(h->tmpU, coeffs, bytes, cudaMemcpyHostToDevice, h->stream));
  return opf_set_state_device(h, (const double*)h->tmpU);
}

int opf_get_state_device(opf_t* h, double* d_coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!d_coeffs) return fail(OPF_EINVAL, "opf_get_state: NULL buffer");
  opf::launch_internal_to_abi(h->d, h->U, (double2*)d_coeffs, 1, h->stream);
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  return OPF_OK;
}

int opf_get_state(opf_t* h, double* coeffs) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!coeffs) return fail(OPF_EINVAL, "opf_get_state: NULL buffer");
  opf::launch_internal_to_abi(h->d, h->U, h->abi, 1, h->stream);
  CU(cudaMemcpyAsync(coeffs, h->abi, 3 * (size_t)h->d.F * sizeof(double2), cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  return OPF_OK;
}

int opf_step(opf_t* h, int n) {
  if (check_handle(h)) return OPF_EINVAL;
  if (n < 0) return fail(OPF_EINVAL, "opf_step: n < 0");
  for (int s = 0; s < n; ++s) {
    h->nslots = 0;
    if (h->use_graph) {
      if (!h->gexec) {
        cudaGraph_t g;
        CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_step(h);
        CU(cudaStreamEndCapture(h->stream, &g));
        h->graph_nslots = h->nslots;
        cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          h->gexec = nullptr;
          return fail(OPF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
      }
      CU(cudaGraphLaunch(h->gexec, h->stream));
      h->nslots = h->graph_nslots;  // event nodes captured with the graph
    } else {
      enqueue_step(h);
    }
    if (h->timing) {
      CU(cudaStreamSynchronize(h->stream));
      int rc = harvest_timing(h);
      if (rc) return rc;
    }
  }
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  h->time += n * h->d.dt;
  return OPF_OK;
}

int opf_energy(opf_t* h, double out[3]) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!out) return fail(OPF_EINVAL, "opf_energy: NULL out");
  opf::launch_curl(h->d, h->ds, h->U, h->W6, h->stream);
  opf::launch_energy(h->d, h->ds, h->U, h->W6, h->beta_p, h->partial, h->nblk_energy, h->out3,
                     h->stream);
  CU(cudaMemcpyAsync(out, h->out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  if (!std::isfinite(out[0]) || !std::isfinite(out[1]) || !std::isfinite(out[2]))
    return fail(OPF_ENAN, "opf_energy: non-finite state");
  return OPF_OK;
}

int opf_wall_residual(opf_t* h, double out[2]) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!out) return fail(OPF_EINVAL, "opf_wall_residual: NULL out");
  opf::launch_wall(h->d, h->ds, h->U, h->out2, h->stream);
  CU(cudaMemcpyAsync(out, h->out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  return OPF_OK;
}

int opf_nonlinear(opf_t* h, const double* coeffs, double* out) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!coeffs || !out) return fail(OPF_EINVAL, "opf_nonlinear: NULL buffer");
  const size_t bytes = 3 * (size_t)h->d.F * sizeof(double2);
  CU(cudaMemcpyAsync(h->abi, coeffs, bytes, cudaMemcpyHostToDevice, h->stream));
  opf::launch_abi_to_internal(h->d, h->abi, h->tmpU, h->stream);
  const int timing = h->timing;
  h->timing = 0;
  enqueue_nonlinear(h, h->tmpU, h->Nq);
  h->timing = timing;
  opf::launch_internal_to_abi(h->d, h->Nq, h->abi, 1, h->stream);
  CU(cudaMemcpyAsync(out, h->abi, bytes, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaGetLastError());
  return OPF_OK;
}

int opf_set_option(opf_t* h, const char* key, double v) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!key) return fail(OPF_EINVAL, "opf_set_option: NULL key");
  if (!strcmp(key, "precision")) {
    if (v != 0.0 && v != 1.0) return fail(OPF_EINVAL, "precision: 0 (FP64) or 1 (mixed)");
    h->precision = (int)v;
  } else if (!strcmp(key, "n_corr")) {
    if (!(v >= 1 && v <= 16 && v == std::floor(v))) return fail(OPF_EINVAL, "n_corr: 1..16");
    h->n_corr = (int)v;
  } else if (!strcmp(key, "graph")) {
    if (v != 0.0 && v != 1.0) return fail(OPF_EINVAL, "graph: 0 or 1");
    h->use_graph = (int)v;
  } else if (!strcmp(key, "timing")) {
    if (v != 0.0 && v != 1.0) return fail(OPF_EINVAL, "timing: 0 or 1");
    h->timing = (int)v;
  } else {
    return fail(OPF_EINVAL, std::string("unknown option ") + key);
  }
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return OPF_OK;
}

int opf_get_option(opf_t* h, const char* key, double* v) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!key || !v) return fail(OPF_EINVAL, "opf_get_option: NULL argument");
  if (!strcmp(key, "precision")) *v = h->precision;
  else if (!strcmp(key, "n_corr")) *v = h->n_corr;
  else if (!strcmp(key, "graph")) *v = h->use_graph;
  else if (!strcmp(key, "timing")) *v = h->timing;
  else return fail(OPF_EINVAL, std::string("unknown option ") + key);
  return OPF_OK;
}

int opf_get_dt(opf_t* h, double* dt) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!dt) return fail(OPF_EINVAL, "NULL out");
  *dt = h->d.dt;
  return OPF_OK;
}

int opf_get_time(opf_t* h, double* t) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!t) return fail(OPF_EINVAL, "NULL out");
  *t = h->time;
  return OPF_OK;
}

int opf_get_beta(opf_t* h, double* beta) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!beta) return fail(OPF_EINVAL, "NULL out");
  double bp = 0.0;
  CU(cudaMemcpyAsync(&bp, h->beta_p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  *beta = bp * h->d.Re / 4.0;
  return OPF_OK;
}

int opf_set_stream(opf_t* h, void* stream) {
  if (check_handle(h)) return OPF_EINVAL;
  CU(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own;
  return OPF_OK;
}

int opf_kernel_times(opf_t* h, int cap, int* count, const char** names, double* total_ms,
                     int* launches, int reset) {
  if (check_handle(h)) return OPF_EINVAL;
  if (!count) return fail(OPF_EINVAL, "NULL count");
  int c = 0;
  for (int i = 0; i < kNumNames && c < cap; ++i) {
    if (names) names[c] = kNames[i];
    if (total_ms) total_ms[c] = h->tot_ms[i];
    if (launches) launches[c] = h->tot_n[i];
    ++c;
  }
  *count = c;
  if (reset)
    for (int i = 0; i < kNumNames; ++i) {
      h->tot_ms[i] = 0;
      h->tot_n[i] = 0;
    }
  return OPF_OK;
}

int opf_setup_query(int N, int K, int M, int m_p, double alpha, double Re, double dt,
                    const char* what, double* out, long cap, long* len) {
  if (N < 9 || K < 1 || M < 1 || m_p < 1 || !(alpha > 0) || !(Re > 0) || !(dt > 0) || !what || !len)
    return fail(OPF_EINVAL, "opf_setup_query: bad arguments");
  opf::Setup s;
  s.N = N;
  s.K = K;
  s.M = M;
  s.m_p = m_p;
  s.alpha = alpha;
  s.Re = Re;
  s.dt = dt;
  s.c = 0.5;
  std::string err;
  if (!opf::build_setup(&s, &err)) return fail(OPF_EINVAL, "opf_setup_query: " + err);
  const std::vector<double>* v = nullptr;
  if (!strcmp(what, "r")) v = &s.r;
  else if (!strcmp(what, "wq")) v = &s.wq;
  else if (!strcmp(what, "d1")) v = &s.d1;
  else if (!strcmp(what, "d2")) v = &s.d2;
  else if (!strcmp(what, "G")) v = &s.G;
  else if (!strcmp(what, "basis")) v = &s.basis;
  else return fail(OPF_EINVAL, std::string("opf_setup_query: unknown array ") + what);
  *len = (long)v->size();
  if (!out) return OPF_OK;
  if (cap < *len) return fail(OPF_EINVAL, "opf_setup_query: output too small");
  std::memcpy(out, v->data(), v->size() * sizeof(double));
  return OPF_OK;
}

}  // extern "C"
