// Internal declarations of libopf: host setup data, device buffers, kernels.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/opf.h"

namespace opf {

constexpr int kStencil = 9;   // 9-point radial finite differences (section 2)
constexpr int kLuSlots = 13;  // per LU row: 8 L entries, 1/U_ii, 4 U entries
constexpr int kMaxRadix = 8;  // FFT plans: at most 8 stages of radix 2/3/4/5

// Mixed-radix plan for one transform length (Stockham, radices 2, 3, 4, 5).
struct FftPlan {
  int n;
  int nst;
  int rad[kMaxRadix];
};

bool make_plan(int n, FftPlan* p);

// ---------------------------------------------------------------- host setup
// Everything the device path needs that does not change during stepping
// (rebuilt only when dt or c changes).  Written independently of the CPU
// oracle: Fornberg recursion for the stencils, pivot-free banded LU.
struct Setup {
  int N = 0, K = 0, M = 0, m_p = 1;
  double alpha = 0, Re = 0, dt = 0, c = 0.5;
  std::vector<double> r_user;  // a user radial mesh (N points), empty = the default points
  std::vector<double> r, rinv;
  std::vector<double> d1;     // [2 parity: 0 even, 1 odd][N][9] first derivative
  std::vector<double> d2;     // same layout, second derivative
  std::vector<double> wq;     // quadrature: sum wq f ~ int_0^1 f r dr (f even)
  int nJ = 0;                 // number of distinct |j| used by Helmholtz operators
  std::vector<int> jidx;      // |j| -> compact index (or -1)
  std::vector<int> hop;       // [M][3] compact |j| index for (m, field u+,u-,u_z)
  std::vector<double> luH;    // [K][nJ][N][13]   Helmholtz (Dirichlet wall row)
  std::vector<double> luP;    // [K*M + 1][N][13] Poisson (Neumann wall row);
                              // the extra last operator is (0,0) with p(1) = 0
  std::vector<double> basis;  // [K][M][6][N] influence-matrix responses
  std::vector<double> ainv;   // [M][2K-1][16][2] inverse influence matrices
  std::vector<double> G;      // fixed-flux response of the (0,0) axial mode
  double flux_G = 0;          // 2 pi sum wq G
  // two-partition (split) factors of the same operators, built when spike is
  // set: per operator N rows of 13 slots (top block, then bottom block), N
  // rows of 4 spike entries, 64 entries of the interface inverse
  bool spike = false;
  std::vector<double> luH2, luP2, spkH, spkP, rH, rP;
};

bool build_setup(Setup* s, std::string* err);

// --------------------------------------------------------------- device side
// Per-trajectory scalars at the head of each trajectory's setup arrays.
constexpr int kPrmRe = 0, kPrmDt = 1, kPrmC = 2, kPrmSumWG = 3, kPrmCi = 4, kPrmCu = 5, kPrmCount = 8;

struct DevSetup {
  double* prm = nullptr;  // [kPrmCount] Re, dt, c, sum(wq G)
  double* rinv = nullptr;
  double* d1 = nullptr;
  double* wq = nullptr;
  int* hop = nullptr;
  double* luH = nullptr;
  double* luP = nullptr;
  double* basis = nullptr;  // device order [K][M][N][6] (host Setup: [K][M][6][N])
  double2* ainv = nullptr;
  double* G = nullptr;
  double2* tw_z = nullptr;   // e^{+2 pi i t / nz}, t < nz
  double2* tw_th = nullptr;  // e^{+2 pi i t / nth}
  float2* tw_z32 = nullptr;
  float2* tw_th32 = nullptr;
  double* r = nullptr;    // radial points (null where the split curl is not used)
  float* d1f = nullptr;   // d1 in FP32, then 1/r in FP32 ([2][N][9] + [N])
  // two-partition (split) solve data (Setup::luH2 ...; null unless built)
  double *luH2 = nullptr, *luP2 = nullptr, *spkH = nullptr, *spkP = nullptr, *rH = nullptr, *rP = nullptr;
};

// Spectral fields are stored [field][m][n][kk] (kk = k + K - 1 fastest).
// Physical-in-z intermediates are stored [field][n][z][m] (m fastest).
struct Dims {
  int N, K, M, m_p, nk, nz, nth;
  double inv_grid;  // 1 / (nz nth): scaling of the forward transforms
  double alpha, Re, dt, c;  // host copies (trajectory 0); kernels read DevSetup::prm
  long F;         // complex values per spectral field = M * N * nk
  int mcz, mca;   // m columns per block: z synthesis, z analysis
  int zc;         // z rows per block in the theta/product kernel
  int tile = 0;   // modes per block in the solve (0: heuristic)
  int spike = 0;  // solve the banded systems in two halves at once (split factors built)
  int fused = 0;  // mixed precision: the three transform kernels as one cluster launch where it
                  // fits (0 off, 1 cluster size chosen, 2/4/8 that cluster size)
  int pdl = 0;    // programmatic dependent launch of the step kernels: 0 off, 1 trigger at
                  // the top of each block, 2 before its final store phase
  // batching: B trajectories of this shape per launch (grid z); trajectory b's
  // work buffers start b*ss bytes after trajectory 0's, its setup arrays b*ps
  // bytes after (ps = 0: one shared setup)
  int B = 1;
  long ss = 0, ps = 0;
  const double* prm = nullptr;  // trajectory 0's DevSetup::prm
  // CFL reduction in the product kernel (null: off): per-trajectory maximum of
  // |u_r|/dr, |u_t|/(r dtheta), |u_z|/dz written at cfl (+ b*ss), radial
  // points from rinv_cfl (+ b*ps)
  double* cfl = nullptr;
  const double* rinv_cfl = nullptr;
  // frame rotation Omega (Cartesian, pipe axis z): Coriolis force -2 Omega x u
  // added to the nonlinear term in the product kernel (rotate: any non-zero)
  int rotate = 0;
  double rot_x = 0.0, rot_y = 0.0, rot_z = 0.0;
  // constant body force in the internal +- layout [3][m][n][kk] added to the
  // nonlinear term after truncation (null: none)
  const double2* forcing = nullptr;
};

void choose_chunks(Dims* d);
bool prepare_kernel_attrs(const Dims& d);
bool prepare_nonlinear_attrs(const Dims& d);  // FP64 nonlinear-term kernels only
// Shared memory a launch shape needs (autotuner candidates must fit).
size_t zsynth_smem(const Dims& d, int mc, size_t vb);
size_t zanalysis_smem(const Dims& d, int mc, size_t vb);
size_t product_smem(const Dims& d, int zc, size_t vb);
size_t solve_smem_bytes(int N, int T);
void set_last_error(const std::string& m);  // text returned by opf_last_error()

// Launch wrappers (kernels live in opf_kernels.cu).
// (flag: skip the conversion where the NaN check before it set *flag; beta: reset to 0;
// nan_out: set where a coefficient read is not finite; herm: two words, zeroed by the
// caller, that receive the m = 0 asymmetry and magnitude maxima)
void launch_abi_to_internal(const Dims& d, const double2* abi, double2* U, cudaStream_t st,
                            const int* flag = nullptr, double* beta = nullptr, int* nan_out = nullptr,
                            unsigned* herm = nullptr);
void launch_copy_unless(const double2* src, double2* dst, long n, const int* flag, double* beta,
                        cudaStream_t st);
void launch_internal_to_abi(const Dims& d, const double2* U, double2* abi, int components_rtz,
                            cudaStream_t st);
void launch_curl(const Dims& d, const DevSetup& s, const double2* U, double2* W6, cudaStream_t st);
void launch_zsynth(const Dims& d, const DevSetup& s, const FftPlan& pz, const double2* W6,
                   double2* Z6, cudaStream_t st);
void launch_product(const Dims& d, const DevSetup& s, const FftPlan& pth, const double2* Z6,
                    double2* ZN, cudaStream_t st);
void launch_zanalysis(const Dims& d, const DevSetup& s, const FftPlan& pz, const double2* ZN,
                      double2* Nout, cudaStream_t st);
// Mixed precision (FP32 transforms and product of the perturbation, FP64
// terms linear in it): curl with base-flow split, then the FP32 transforms.
void launch_curl_split32(const Dims& d, const DevSetup& s, const double2* U, float2* W6,
                         double2* Nlin, cudaStream_t st);
void launch_zsynth32(const Dims& d, const DevSetup& s, const FftPlan& pz, const float2* W6,
                     float2* Z6, cudaStream_t st);
void launch_product32(const Dims& d, const DevSetup& s, const FftPlan& pth, const float2* Z6,
                      float2* ZN, cudaStream_t st);
void launch_zanalysis32(const Dims& d, const DevSetup& s, const FftPlan& pz, const float2* ZN,
                        const double2* Nlin, double2* Nout, cudaStream_t st);
// The three FP32 transform kernels above as one cluster launch (false, and
// nothing launched, where the shape takes the three-kernel path).
bool launch_nl_fused32(const Dims& d, const DevSetup& s, const float2* W6, const double2* Nlin, double2* Nout,
                       cudaStream_t st);
int fused32_cluster(const Dims& d);
struct SolveArgs {
  const double2* Uj;
  const double2* Na;
  const double2* Nb;
  double wa, wb;
  double2* Uout;
  double* beta_p;  // device scalar: beta' of this solve (written by the (0,0) mode)
  // curl of the solved state for the next nonlinear evaluation, computed by
  // the same blocks from their radial columns: 0 none, 1 FP64 into W6
  // (double2), 2 mixed precision into W6 (float2) and the FP64 linear terms Nlin
  int curl = 0;
  void* W6 = nullptr;
  double2* Nlin = nullptr;
};
void launch_solve(const Dims& d, const DevSetup& s, const SolveArgs& a, int nJ, cudaStream_t st);
void launch_energy(const Dims& d, const DevSetup& s, const double2* U, const double2* W6,
                   const double* beta_p, double* partial, int nblk, double* out3, cudaStream_t st);
int energy_blocks(const Dims& d);
void launch_wall(const Dims& d, const DevSetup& s, const double2* U, double* out2, cudaStream_t st);
void launch_nan_check(const double* x, long n, int* flag, cudaStream_t st);

// Tensor-core GEMM (tcgen05, BF16 operands, FP32 accumulation):
// C[m][n] = sum_k A[m][k] B[n][k] for m < M, n < N; A [Mp][Kp] and B [Np][Kp]
// row-major BF16, zero padded (Mp, Np multiples of 128, Kp of 64), 16-byte
// aligned.  Epilogue per (m, n): x = C + bias[n]; pre_f32 = x; x = gelu(x)
// if gelu; out_f32 = x (+= x if accumulate); out_bf16 = bf16(x); outputs
// have row stride ldo.  d_err (device int) is set on a timed-out wait.
// work (device, work_floats floats; may be null) lets plain FP32 outputs (no
// bias, GELU or BF16 copy) split K across CTAs; the partial sums are added in
// a fixed order, so results do not depend on scheduling.
struct TcEpilogue {
  const float* bias;
  int gelu;
  float* pre_f32;
  float* out_f32;
  int accumulate;
  void* out_bf16;
  long ldo;
};
int tc_gemm(const void* A, const void* B, int M, int N, int Mp, int Np, int Kp, const TcEpilogue& e, int* d_err,
            cudaStream_t st, float* work = nullptr, long work_floats = 0);

}  // namespace opf
