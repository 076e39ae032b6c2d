// msd_internal.h -- shared declarations of the libmsd CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "msd.h"

namespace msd {

constexpr int MAXK = MSD_MAX_ORDER;
constexpr int NCH = 5;  // channels: value, d/dx, d/dy, d/dz, laplacian

enum StatusBits : int { ST_SINGULAR = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

// Bytes of one excitation record of order k: k hole bytes, k particle bytes, padded to a
// power of two so one vector load fetches it.
__host__ __device__ constexpr int rec_bytes(int k) {
    return k <= 1 ? 2 : k == 2 ? 4 : k <= 4 ? 8 : 16;
}

// Excitation strings of one spin on the device, grouped by order.  Internal index i of
// order k lies in [goff[k], goff[k+1]); group 0 holds the reference.  Group k >= 1 (unless
// dense) is a whole number of warp batches of kBatch records starting at byte roff[k] of rec;
// the lane-l record of a batch is the string that lane l handles, and no two records of a batch
// share the residue mod 32 of the particle in any one slot.  Unused slots hold records filled
// with kEmptyRecord bytes and carry C = 0; their first hole byte 0xFF is no valid hole (a spin
// with 255 or more electrons is rejected: its A_0^{-1} would not fit in shared memory).  With dense1 set the singles occupy a
// dense n x m block (index goff[1] + h m + p; absent singles carry C = 0) and have no records.
constexpr int kBatch = 32;
constexpr uint8_t kEmptyRecord = 0xFF;
struct ExcDev {
    int n_exc = 0;
    int kmax = 0;
    int dense1 = 0;
    int goff[MAXK + 2] = {0};
    long long roff[MAXK + 2] = {0};
    const uint8_t* rec = nullptr;
};

// Kernel launch wrappers (msd_kernels.cu).  Template parameter pairs are selected at
// run time by `mixed`: FP64 everywhere, or FP32 orbitals/table/excitations.
struct Launch {
    cudaStream_t stream;
    int* status;             // device status word
    long long* launches;     // host counter of kernel launches (nullable)
    cudaEvent_t t0 = nullptr;  // recorded before/after the excitation-sweep kernel (nullable)
    cudaEvent_t t1 = nullptr;
    void count(int k = 1) const {
        if (launches) *launches += k;
    }
};

// Orbitals phi^a_j at P points.  Point p belongs to walker p / ppw and sits at
// pos + (p / ppw) * wstride + (p_off + p % ppw) * 3.  out[p][a][j], a < nch (1 or 5).
void launch_orbitals(const Launch& L, bool mixed, int nch, int P, int ppw, const double* pos,
                     long long wstride, int p_off, const double4* bas, const int8_t* blm, int nb,
                     const void* B, int N, void* out);

// The same orbitals on the tensor cores (FP32 path, msd_tc.cu): B of one spin split on
// the host into three TF32 pieces in the operand layout the kernel copies (tc_split_B), TN <= 256
// columns per tile, nT column tiles, nK chunks of 8 basis functions; out is FP32.
struct TcPlan {
    int nT = 0, TN = 0, nK = 0;
    size_t floats = 0;  // size of the split B
    size_t smem = 0;    // dynamic shared memory per block
};
TcPlan tc_plan(int nb, int N);
void tc_split_B(const TcPlan& t, int nb, int N, const double* B, float* out);
// basf [nb][2] float4: (centre hi, alpha), (centre lo, 0) from centres [nb][3] and exponents [nb].
void tc_basis_pairs(int nb, const double* centers, const double* alpha, float* out);
void launch_orbitals_tc(const Launch& L, int nch, int P, int ppw, const double* pos, long long wstride, int p_off,
                        const float4* basf, const int8_t* blm, int nb, const TcPlan& t, const float* Bsplit, int N,
                        float* out);

// T[w] = Ainv[w] * Phi[w][:, n:N] on the tensor cores (FP32 path; n <= 256, table_tc_supported).
bool table_tc_supported(int n);
void launch_table_tc(const Launch& L, int W, int n, int N, const double* Ainv, const float* Phi, float* T);

// One block that waits limit_ns on an mbarrier nothing completes and sets ST_TIMEOUT (a check of the
// bounded-wait failure path).
void launch_wait_selftest(const Launch& L, unsigned long long limit_ns);

// Gauss-Jordan inverse with partial pivoting of A_0 = Phi[w][:, :n] for every walker; cond (nullable)
// receives ||A_0||_inf ||A_0^{-1}||_inf per walker.
void launch_inverse(const Launch& L, bool mixed, int W, int n, int N, const void* Phi, double* Ainv,
                    double* logdet, double* sgn, double* cond = nullptr);

// T[w] = Ainv[w] * Phi[w][:, n:N].
void launch_table(const Launch& L, bool mixed, int W, int n, int N, const double* Ainv, const void* Phi,
                  void* T);

// t[w][i] = det T_i (value of every excitation ratio, Section III).
void launch_exc_det(const Launch& L, bool mixed, int W, int n, int m, const ExcDev& g, const void* T, void* t);

// C[w][u] = sum_{I in terms(u)} c_I t_other[w][other_I].  The light kernel skips strings with
// more than heavy_threshold() terms; the heavy kernel reduces those with a block each.
void launch_ci_contract(const Launch& L, bool mixed, int W, int n_exc, int n_exc_other, const int* off,
                        const int* other, const double* c, const void* t_other, void* C);
void launch_ci_contract_heavy(const Launch& L, bool mixed, int W, int n_exc, int n_exc_other, int n_heavy,
                              const int* heavy, const int* off, const int* other, const double* c,
                              const void* t_other, void* C);
int heavy_threshold();

// S[w] = sum_u C[w][u] t[w][u] in FP64.
void launch_ci_dot(const Launch& L, bool mixed, int W, int n_exc, const void* C, const void* t, double* S);

struct RatioArgs {
    int W, n, N, m, row, nch;
    const void* phi;       // [W][nch][N] orbitals at the evaluated position
    const double* Ainv;    // [W][n][n]
    const void* T;         // [W][n][m]
    const void* C;         // [W][n_exc]
    const double* S;       // [W]
    ExcDev g;
    double* ratio; long long rs;   // ratio[w * rs]
    double* grad; long long gs;    // grad[w * gs + a]
    double* lap; long long ls;     // lap[w * ls]
    double* rho;           // [W] saved proposal (nullable)
    double* num;           // [W][NCH] saved proposal (nullable)
    void* y0;              // [W][m] saved proposal (nullable)
};
void launch_ratio(const Launch& L, bool mixed, const RatioArgs& a);

struct AcceptArgs {
    int W, n, N, m, row, elec, n_tot;
    const uint8_t* accept;
    const void* phi;       // [W][nch][N], channel 0 = values at r'
    int nch;
    const double* rho;
    const double* num;     // [W][NCH]
    const void* y0;        // [W][m]
    const double* rnew;    // [W][3]
    double* Ainv;
    void* T;
    double* R;
    double* logdet;
    double* sgn;
    double* S;
    const int* skip = nullptr;  // [W] walkers held elsewhere (>= 0): their flags are not raised (nullable)
};
void launch_accept(const Launch& L, bool mixed, const AcceptArgs& a);

void launch_propose(const Launch& L, int W, int n_tot, int elec, const double* R, const double* eta, double tau,
                    double* rnew);
// Rows of walkers in and out of the FP64 rescue context: dst[s][:] = src[map[s]][:] (gather, every
// slot) and dst[map[s]][:] = src[s][:] for s < n_real (scatter).
void launch_gather_rows(const Launch& L, int n_slots, const int* map, int row, const double* src, double* dst);
void launch_gather_bytes(const Launch& L, int n_slots, const int* map, const uint8_t* src, uint8_t* dst);
void launch_scatter_rows(const Launch& L, int n_real, const int* map, int row, const double* src, double* dst);
// ST_NONFINITE if any of ratio[0..W) is not finite.
void launch_check_finite(const Launch& L, int W, const double* ratio);
struct BatchPlan;
// The same for a batch: a non-finite ratio of walker w flags its system's status.
void launch_check_finite_batched(const Launch& L, const BatchPlan& P, int W, const double* ratio);
void launch_metropolis(const Launch& L, int W, const double* u, const double* ratio, uint8_t* accept);
void launch_state(const Launch& L, int W, const double* ld0, const double* sg0, const double* ld1,
                  const double* sg1, const double* S, double* logabs, double* sign);

size_t ratio_smem_bytes(bool mixed, int n, int m, int nch);

// Batched systems in single launches: per-system descriptors (device), built by the host at
// initialisation.  A kernel reads its system, derives the moving electron e = t mod n_tot and
// its spin, and runs the single-system per-block code on that system's arrays.
struct OrbArgs {
    const double4* bas;
    const int8_t* blm;
    int nb;
    const void* B;   // [nb][N] of the spin
    int N;
    void* out;       // [W][nch][N] orbitals at the proposed positions
    const float* Bsplit;  // FP32 path: B in TF32 pieces for the tensor cores (TcPlan of the spin)
    int TN, nT;
    const float4* basf;   // FP32 path: basis centres as (hi, lo) pairs (tc_basis_pairs)
};
struct BatchSys {
    int n_tot, n_up, W, w_off;  // electrons, walkers, offset of the walkers in concatenated arrays
    int* status;                // the system's status word
    int* ratio_status;          // where the ratio launch reports instead (nullable: status)
    const double* R;            // [W][n_tot][3]
    OrbArgs orb[2];             // per spin
    RatioArgs ratio[2];         // per spin, without row, nch and outputs
    AcceptArgs accept[2];       // per spin, without row, elec, nch, accept flags and rnew
};
struct BatchPlan {
    const BatchSys* sys = nullptr;
    int n_sys = 0;
    const int2* blk = nullptr;  // ratio and accept blocks: (system, walker), grouped by ratio_groups
    int n_blk = 0;
    // ratio launches: blocks [gfirst[i], gfirst[i + 1]) share a shared-memory size gsmem[i], so
    // small systems are not held to the occupancy of the largest one
    static constexpr int kMaxGroups = 4;
    int n_groups = 0;
    int gfirst[kMaxGroups + 1] = {0};
    size_t gsmem[kMaxGroups] = {0};
    const int4* tiles = nullptr;  // orbital tiles: (system, first point, first orbital, -)
    int n_tiles = 0;
    const int* wsys = nullptr;  // system of each concatenated walker
    size_t ratio_smem = 0, accept_smem = 0;
    // FP32 path: tensor-core orbital tiles (system, point tile of 25, column tile, -) and their
    // shared memory (the largest any system needs)
    const int4* tc_tiles = nullptr;
    int n_tc_tiles = 0;
    size_t tc_smem = 0;
    // the fused Metropolis step (launch_step_batched): (system, walker) items per group, ordered by
    // decreasing cost, the group's shared memory and a pair of counters per group (zero between launches)
    const int2* items = nullptr;
    size_t step_smem[kMaxGroups] = {0};
    int* counters = nullptr;
};
// One Metropolis step of group `group`'s walkers as one persistent launch of `grid` blocks.
void launch_step_batched(const Launch& L, bool mixed, const BatchPlan& P, int group, int grid, int t,
                         const double* eta, double tau, const double* u, double* ratio, double* grad, double* lap,
                         uint8_t* accept, double* rnew);
// Blocks of the step kernel an SM holds with `smem` bytes of shared memory.
int step_blocks_per_sm(bool mixed, size_t smem);
void launch_orbitals_batched(const Launch& L, bool mixed, const BatchPlan& P, int t, int nch, const double* rnew);
void launch_orbitals_tc_batched(const Launch& L, const BatchPlan& P, int t, int nch, const double* rnew);
int tc_tile_points(int nch);  // points per tensor-core tile for 1 or 5 channels
void launch_ratio_batched(const Launch& L, bool mixed, const BatchPlan& P, int t, int nch, double* ratio, double* grad,
                          double* lap);
void launch_accept_batched(const Launch& L, bool mixed, const BatchPlan& P, int t, int nch, const uint8_t* accept,
                           const double* rnew);
void launch_propose_batched(const Launch& L, const BatchPlan& P, int W_total, int t, const double* eta, double tau,
                            double* rnew);
size_t accept_smem_bytes(int n);
int orbital_tile_points();
int orbital_tile_orbitals();

// The canonical method (msd_kernels.cu): D[w][j] = A_j^{-1} ([c][r]) and t[w][j] = det A_j / det A_0
// of every string j, the row-replacement ratios ru[w][j] of a proposal, their update on accept.
void launch_canon_build(const Launch& L, int W, int n, int N, int m, const ExcDev& g, const double* Phi,
                        const uint8_t* used, const double* ld0, const double* sg0, double* D, double* t);
void launch_canon_ratio(const Launch& L, int W, int n, int N, int m, int row, int nch, const ExcDev& g,
                        const uint8_t* used, const double* phi, const double* D, const double* t, const double* C,
                        const double* S, double* ru, double* ratio, double* grad, double* lap, double* num,
                        double* rho);
void launch_canon_accept(const Launch& L, int W, int n, int N, int m, int row, int elec, int n_tot, const ExcDev& g,
                         const uint8_t* used, const uint8_t* accept, const double* phi_new, int nch, double* Phi,
                         double* D, double* t, const double* ru, const double* rnew, double* R, const double* rho,
                         const double* num, double* logdet, double* sgn, double* S);

// Adjoint of log|Psi| (msd_backward.cu).  dci[I] += sum_w gbar[w] t0[w][iu[I]] t1[w][id[I]] / S[w].
void launch_dci(const Launch& L, bool mixed, int W, long long n_det, const int* iu, const int* id, const double* gbar,
                const double* S, const void* t0, int ld0, const void* t1, int ld1, double* dci);
// M[w] (n x N, FP64) <- gbar[w] Ainv[w]^T [I - Tbar T^T | Tbar], Tbar = (1/S) sum_u C_u cof(T_u).
size_t tbar_smem_bytes(bool mixed, int n, int m);
void launch_phibar(const Launch& L, bool mixed, int W, int n, int m, int N, const ExcDev& g, const void* T,
                   const void* C, const double* S, const double* Ainv, const double* gbar, double* M);
// Tbar = (1/S) sum_u C_u cof(T_u) into columns n..N-1 of M (n x N, FP64).
void launch_tbar(const Launch& L, bool mixed, int W, int n, int m, int N, const ExcDev& g, const void* T, const void* C,
                 const double* S, double* M);
// grad [W][n_tot][3] and lap [W][n_tot] of the spin's electrons e_off .. e_off + n - 1 from Tbar
// (in M) and the orbitals with derivatives at every electron, phid [W n][5][N].
// G' = A_0^{-T} Tbar goes to Gp [W][n][m] (FP32 on the mixed path, FP64 otherwise); n <= 256.
void launch_all_gradlap(const Launch& L, bool mixed, int W, int n, int m, int N, int n_tot, int e_off,
                        const double* Ainv, const void* T, const double* M, const void* phid, void* Gp, double* grad,
                        double* lap);
// chi[p][mu] (values, FP64) at P points laid out as for launch_orbitals.
void launch_chi(const Launch& L, int P, int ppw, const double* pos, long long wstride, int p_off, const double4* bas,
                const int8_t* blm, int nb, double* chi);
// dB[mu][j] += sum_p chi[p][mu] Phib[p][j].
void launch_dB(const Launch& L, int P, int nb, int N, const double* chi, const double* Phib, double* dB);

// VMC energy driver (msd_vmc.cu): Jastrow factor and local energy, FP64.
struct HamArgs {
    int W, n_tot, n_up, n_nuc;
    const double* R;      // [W][n_tot][3] current positions
    const double4* nuc;   // [n_nuc] (x, y, z, Z)
    double b_ee, b_en;    // Pade parameters of the Jastrow terms (<= 0: term absent)
    double vnn;           // nuclear repulsion sum_{I<J} Z_I Z_J / R_IJ
};
// ratio[w] *= exp(J(R') - J(R)) for the move of electron elec to rnew[w].
void launch_jastrow_ratio(const Launch& L, const HamArgs& a, int elec, const double* rnew, double* ratio);
// eloc[w] and, if parts is non-NULL, parts[w] = (kinetic, V_ee, V_en, V_nn), from grad_i D / D
// [W][n_tot][3] and lap_i D / D [W][n_tot] of the determinant part.
void launch_local_energy(const Launch& L, const HamArgs& a, const double* gradD, const double* lapD, double* eloc,
                         double* parts);

// Fixed device scratch of msd_ratio_noalloc (msd_kernels.cu): its size, and its address on the
// current device (looked up on the first call per device).
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;
cudaError_t noalloc_scratch(void** ptr);

}  // namespace msd
