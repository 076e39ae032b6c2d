/*
 * msd.h -- C ABI of libmsd: the multi-Slater-determinant "table method"
 * (Clark, Morales, McMinis, Kim, Scuseria, arXiv:1106.2456) on one NVIDIA GB300 GPU.
 *
 * Wavefunction (Section II):   Psi(R) = sum_I c_I det M_up,I(R) det M_dn,I(R),
 *   M_s,I(r, c) = phi_{col_I(c)}(r_r)  -- rows are electrons, columns orbitals.
 * Orbitals 0..n_s-1 of spin s form the reference determinant M_s,0; orbitals
 * n_s..N_s-1 are the m_s = N_s - n_s virtuals.  An excitation string of order k
 * replaces the occupied columns h_1 < ... < h_k IN PLACE by the virtual orbitals
 * n_s + p_1 < ... < n_s + p_k (column h_q holds orbital n_s + p_q).
 *
 * Per walker the library keeps, for each spin, A_0^{-1} (FP64) and the excitation
 * table T = A_0^{-1} Phi_virt (Section III, Algorithm 1 step 3), and computes
 *   - the ratio Psi(R') / Psi(R) of a single-electron move (Section II and III):
 *     every excitation ratio det A_u / det A_0 is the k x k determinant of the table
 *     entries T[h_q, p_l] (Section III), bordered by the moved electron's row;
 *   - grad_i Psi / Psi and lap_i Psi / Psi at the proposed position (Section IV-A:
 *     the same table with the electron's row replaced by derivative rows);
 *   - the Sherman-Morrison update of A_0^{-1} and T on acceptance (Section III,
 *     Algorithm 1 step 1), and a from-scratch refresh every refresh_K steps
 *     (Section III: the inverse and determinants recomputed directly).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are DEVICE pointers, read and written in stream order on
 *     the context's CUDA stream; the call returns before the GPU work completes.
 *     Pointers named *_host are HOST pointers; those calls synchronise.
 *   - Arrays are C-contiguous (row-major) with the stated shapes; W = n_walkers.
 *     Walker positions are [W][n_up + n_dn][3] doubles in bohr, up electrons first.
 *   - No call allocates after msd_init, except on first use msd_eval_batch (it creates a
 *     second walker state so that the main one is left untouched), msd_backward,
 *     msd_grad_lap with elec = -1 and msd_local_energy (their workspaces), and
 *     msd_set_hamiltonian (the nuclear charges).
 *   - Device-side numerical faults (a zero or non-finite pivot, a non-finite ratio)
 *     set a status word that msd_sync reports; host-side argument errors return
 *     MSD_ERR_ARG and leave the context unchanged.  msd_last_error explains the
 *     last failure.  No call throws.  A context is used by one host thread at a time.
 */
#ifndef MSD_H
#define MSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSD_MAX_ORDER 8   /* largest per-spin excitation order (Section III: orders stay below 8) */
#define MSD_MAX_ORB 256   /* holes and particles are stored as uint8 */

typedef enum {
    MSD_OK = 0,
    MSD_ERR_ARG = 1,       /* invalid argument; nothing was done */
    MSD_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    MSD_ERR_OOM = 3,       /* device allocation failed */
    MSD_ERR_SINGULAR = 4,  /* a reference determinant or a ratio was zero or not finite */
    MSD_ERR_TIMEOUT = 5,   /* a bounded device wait gave up */
    MSD_ERR_STATE = 6      /* call out of order (e.g. msd_accept without msd_ratio) */
} msd_status;

typedef enum {
    MSD_FP64 = 0,   /* every step in FP64 */
    MSD_MIXED = 1,  /* orbitals, table and excitation determinants in FP32; A_0^{-1},
                       its Sherman-Morrison update, the refresh LU, log|det| and the
                       final CI sums in FP64 */
    MSD_CANONICAL = 2  /* FP64 without the table: every determinant keeps its own inverse,
                       updated by Sherman-Morrison on accept (the method Section III improves
                       on; for comparison).  msd_set_positions, msd_ratio, msd_accept,
                       msd_propose, msd_metropolis, msd_get_state, msd_sync only; memory
                       W x strings x n^2 doubles per spin. */
} msd_precision;

/*
 * Problem description (host arrays, copied by msd_init; the caller keeps ownership).
 * Basis functions are unnormalised Cartesian Gaussians (r - A)^l exp(-alpha |r - A|^2)
 * with l <= 1; phi_j(r) = sum_mu chi_mu(r) B_s[mu][j].
 */
typedef struct {
    int32_t n_elec[2];            /* electrons per spin (n_up, n_dn), each 1..MSD_MAX_ORB */
    int32_t n_orb[2];             /* orbitals per spin N_s >= n_s, N_s - n_s <= MSD_MAX_ORB */
    int32_t n_nuc;
    const double* nuc_xyz;        /* [n_nuc][3] bohr */
    int32_t n_basis;
    const int32_t* bas_center;    /* [n_basis] nucleus index */
    const int8_t* bas_lm;         /* [n_basis] 0 = s, 1 = px, 2 = py, 3 = pz */
    const double* bas_alpha;      /* [n_basis] exponent > 0 */
    const double* B[2];           /* per spin [n_basis][n_orb[s]]; B[1] == B[0] allowed */
    int32_t n_exc[2];             /* unique excitation strings per spin, >= 1 */
    const int32_t* exc_off[2];    /* [n_exc + 1] CSR offsets; string u has order
                                     exc_off[u+1] - exc_off[u] <= MSD_MAX_ORDER;
                                     string 0 must be the reference (order 0) */
    const uint8_t* exc_holes[2];  /* strictly ascending occupied indices < n_elec[s] */
    const uint8_t* exc_parts[2];  /* strictly ascending virtual indices < n_orb[s] - n_elec[s] */
    int64_t n_det;                /* number of terms I, >= 1 */
    const int32_t* det_up;        /* [n_det] spin-up string of term I */
    const int32_t* det_dn;        /* [n_det] spin-down string of term I */
    const double* ci;             /* [n_det] c_I */
    int32_t n_walkers;            /* W >= 1 */
    msd_precision prec;
    int32_t refresh_K;            /* recompute A_0^{-1} and T of a spin from scratch after
                                     this many proposed moves of that spin (>= 1) */
    void* cuda_stream;            /* cudaStream_t for all work; NULL = legacy default stream */
} msd_problem;

typedef struct msd_ctx msd_ctx;

/* Create a context.  n_systems == 1: prob points to one problem; msd_init validates every
 * array, groups the excitation strings by order and packs each order into batches of 32 for
 * the device (msd_describe_records), and allocates all per-walker state.
 * n_systems > 1 (batched uneven systems): prob points to n_systems problems, each with its own
 * electrons, orbitals, strings, terms and walkers (the paper treats one system; running many
 * at once is a throughput concern).  Every per-walker array of every call is then the
 * concatenation over systems in order (walkers of system 0, then of system 1, ...; positions
 * [W_s][n_tot_s][3] per system; msd_backward's dci and dB likewise), and `elec` means electron
 * (elec mod n_tot_s) of system s.  Systems run on internal streams forked from and joined
 * back into the stream of prob[0], so the caller's stream orders every call as usual.
 * msd_copy_state, msd_exc_histogram and msd_ratio_noalloc take single-system contexts only.
 * *out is NULL on failure; the message names the failing system. */
msd_status msd_init(const msd_problem* prob, int32_t n_systems, msd_ctx** out);

/* Validate a problem and report, without any CUDA call, the device layout msd_init would
 * build: for spin s, out[16 s + 0] = internal string count (singles may form a dense n x m
 * block), [1] = 1 if they do, [2] = largest order, [3] = strings whose CI weight sums more
 * than a threshold number of terms, [4] = bytes of excitation records, [5 .. 14] = first
 * internal index of each order 0..8 and the end, [15] = terms referenced.  out has 32 entries. */
msd_status msd_describe(const msd_problem* prob, int64_t* out);

/* The device excitation records of spin `spin` that msd_init would build, without any CUDA
 * call.  Records of order k >= 1 (k = 1 only when the singles are not a dense block) start at
 * byte out_off[k] (out_off has MSD_MAX_ORDER + 2 entries; out_off[MSD_MAX_ORDER + 1] = total
 * bytes) and come in batches of 32, one record per internal string: k hole bytes, then k
 * particle bytes, padded to 2, 4, 8 or 16 bytes (orders 1, 2, 3-4, 5-8).  A record whose
 * first byte is 0xFF is an empty slot.  Within a batch the particles in any one slot have
 * distinct residues mod 32; within a record holes and particles may be permuted with equal
 * parity (Section III: det T_u is unchanged).  out may be NULL to query the size; otherwise
 * it must hold `cap` bytes and receives min(cap, total) bytes; *bytes = total. */
msd_status msd_describe_records(const msd_problem* prob, int32_t spin, uint8_t* out, int64_t cap, int64_t* out_off,
                                int64_t* bytes);

/* Set the walker positions R_dev [W][n_tot][3] and build the state from scratch:
 * orbitals, LU of A_0 (A_0^{-1}, log|det A_0|, sign), T = A_0^{-1} Phi_virt and the CI
 * sums (Section III: initial inverse and determinants computed from scratch). */
msd_status msd_set_positions(msd_ctx* ctx, const double* R_dev);

/* Propose moving electron `elec` (0..n_tot-1) of every walker to rnew_dev [W][3].
 * Writes ratio_dev [W] = Psi(R') / Psi(R) and, if non-NULL, grad_dev [W][3] =
 * grad_elec Psi(R') / Psi(R') and lap_dev [W] = lap_elec Psi(R') / Psi(R') (both at the
 * proposed position).  grad_dev and lap_dev must be both NULL or both non-NULL.  No
 * walker state changes; the proposal is kept for msd_accept.  Runs Algorithm 1 in the
 * bordered form: one table-row contraction y = phi_virt(r') - T^T phi_occ(r') per
 * channel and one (k+1) x (k+1) bordered determinant per excitation and channel. */
msd_status msd_ratio(msd_ctx* ctx, int32_t elec, const double* rnew_dev, double* ratio_dev,
                     double* grad_dev, double* lap_dev);

/* Apply the last msd_ratio proposal (which must be for `elec`) to the walkers whose
 * accept_dev [W] byte is non-zero: Sherman-Morrison update of A_0^{-1} (FP64), rank-1
 * update of T, log|det A_0| and sign, the stored CI sum, and the position. */
msd_status msd_accept(msd_ctx* ctx, int32_t elec, const uint8_t* accept_dev);

/* grad_elec Psi / Psi [W][3] and lap_elec Psi / Psi [W] at the current positions.
 * elec = -1 evaluates every electron: grad_dev [W][n_tot][3], lap_dev [W][n_tot], from one
 * cofactor scatter per spin (the G of a move of electron i is A_0^{-T} Tbar, row i) instead
 * of one sweep per electron. */
msd_status msd_grad_lap(msd_ctx* ctx, int32_t elec, double* grad_dev, double* lap_dev);

/* From scratch at positions R_dev [W][n_tot][3], without touching the walker state:
 * log|Psi| [W], sign [W], and if non-NULL all-electron grad [W][n_tot][3] and
 * lap [W][n_tot] (ratios of Psi, as in msd_grad_lap). */
msd_status msd_eval_batch(msd_ctx* ctx, const double* R_dev, double* logabs_dev, double* sign_dev,
                          double* grad_dev, double* lap_dev);

/* Current walker state: positions R_dev [W][n_tot][3] (may be NULL), log|Psi| [W] and
 * sign [W] (may be NULL), tracked through accepted moves. */
msd_status msd_get_state(msd_ctx* ctx, double* R_dev, double* logabs_dev, double* sign_dev);

/* Copy one piece of the per-walker state to dst_dev (device memory, stream-ordered), for
 * checkpoints and diagnostics.  item: 0 = positions [W][n_tot][3] f64 (spin ignored),
 * 1 = A_0^{-1} [W][n][n] f64 (A^{-1}[c][r]), 2 = table T [W][n][m], 3 = log|det A_0| [W] f64,
 * 4 = sign of det A_0 [W] f64, 5 = S = Psi / (det A_up,0 det A_dn,0) [W] f64 (spin ignored),
 * 6 = CI weights C [W][n_exc], 7 = excitation values t [W][n_exc]; the last msd_ratio
 * proposal (spin ignored): 8 = rho [W] f64, 9 = sum_u C_u d^a_u [W][5] f64,
 * 10 = y^0 [W][m of the moved spin], 11 = orbitals at r' [W][1 or 5][N of the moved spin].
 * T, C, t, y^0 and the orbitals are f64 in MSD_FP64 and f32 in MSD_MIXED; C and t follow the
 * library's internal string order and are only current right after the call that used
 * them.  Returns the byte count in *bytes. */
msd_status msd_copy_state(msd_ctx* ctx, int32_t item, int32_t spin, void* dst_dev, int64_t* bytes);

/* Metropolis helpers of a VMC driver (Section II: a step moves one electron).
 * msd_propose: rnew_dev [W][3] = R[w][elec] + tau * eta_dev [W][3].
 * msd_metropolis: accept_dev [W] = (u_dev[w] < ratio_dev[w]^2) -- no Jastrow factor. */
msd_status msd_propose(msd_ctx* ctx, int32_t elec, const double* eta_dev, double tau, double* rnew_dev);
msd_status msd_metropolis(msd_ctx* ctx, const double* u_dev, const double* ratio_dev, uint8_t* accept_dev);

/* One Metropolis step of every walker (Section II: a step moves one electron): the proposal
 * r' = R[w][elec] + tau * eta_dev[w], ratio_dev [W], grad_dev [W][3] and lap_dev [W] at r' as
 * msd_ratio gives them, the decision accept_dev[w] = (u_dev[w] < ratio_dev[w]^2) (no Jastrow
 * factor), and msd_accept of it.  Every pointer is required.  A single-system context runs the
 * separate calls.  A batched context (elec = electron elec mod n_tot_s of system s) runs the
 * bookkeeping of msd_ratio, then ONE persistent launch per shared-memory group of systems.  Its
 * blocks take (system, walker) items from a device counter, largest systems first, and do the whole
 * step per walker: proposal, orbitals at r' (SIMT, in the path's precision), sweep, decision and
 * update.  The first calls on a batch time three grid sizes per group with CUDA events (and
 * synchronise); later calls use the fastest.  A batch with walkers held in FP64 (msd_set_rescue)
 * runs the separate calls. */
msd_status msd_step(msd_ctx* ctx, int32_t elec, const double* eta_dev, double tau, const double* u_dev,
                    double* ratio_dev, double* grad_dev, double* lap_dev, uint8_t* accept_dev);

/* Host-buffer twins of one walker-move, for callers without device memory: copy the
 * inputs to the device, run, copy the results back, synchronise.
 * msd_ratio_host: rnew_host [W][3] -> ratio_host [W], grad_host [W][3], lap_host [W].
 * msd_accept_host: accept_host [W] bytes. */
msd_status msd_ratio_host(msd_ctx* ctx, int32_t elec, const double* rnew_host, double* ratio_host,
                          double* grad_host, double* lap_host);
msd_status msd_accept_host(msd_ctx* ctx, int32_t elec, const uint8_t* accept_host);

/* Change the CUDA stream used by later calls (cudaStream_t; NULL = legacy default). */
msd_status msd_set_stream(msd_ctx* ctx, void* cuda_stream);

/* Wait for the context's stream; report and clear the device status word. */
msd_status msd_sync(msd_ctx* ctx);

/* Human-readable description of the last failure of this context ("" if none).
 * With ctx == NULL: the last msd_init failure of the calling thread. */
const char* msd_last_error(const msd_ctx* ctx);

/* Counts used by the benchmark's work model: out[0] = n_exc of spin s, out[1 + k] =
 * number of strings of order k (k = 0..MSD_MAX_ORDER) of spin s. */
msd_status msd_exc_histogram(const msd_ctx* ctx, int32_t spin, int64_t* out);

/* Kernel timing for measurement.  msd_timing_start clears the counters and, from then on,
 * brackets every launch of the excitation-sweep kernel (the one that runs steps A2-A5 of
 * msd_ratio) with CUDA events on the context's stream and counts every kernel the library
 * launches.  msd_timing_stop synchronises the stream, stops recording and returns the summed
 * event time of those sweep launches (ms), their number, and the number of all kernel
 * launches since msd_timing_start.  Any output pointer may be NULL. */
msd_status msd_timing_start(msd_ctx* ctx);
msd_status msd_timing_stop(msd_ctx* ctx, double* sweep_ms, int64_t* sweep_launches, int64_t* all_launches);
/* Amortised work inside the window of the last msd_timing_start: out[0] = from-scratch refreshes
 * of a spin (Section III: inverse and table recomputed, every refresh_K moves of that spin),
 * out[1] = CI contractions (the weights C_s of the moving spin recomputed after the other spin
 * changed).  Batched contexts sum over their systems.  Host-side counters; no CUDA call.
 * MSD_ERR_ARG for a NULL argument. */
msd_status msd_timing_counts(const msd_ctx* ctx, int64_t* out);

/* Adjoint of log|Psi| at the current positions, summed over walkers with weights gbar_dev [W]:
 * dci_dev [n_det] = sum_w gbar[w] d log|Psi_w| / d c_I and dB_dev = sum_w gbar[w]
 * d log|Psi_w| / d B_s for each spin, laid out as B_up [n_basis][n_orb[0]] followed by
 * B_dn [n_basis][n_orb[1]] (a restricted B that the caller shares between spins gets the sum
 * of the two blocks).  Both outputs are overwritten.  The paper gives no parameter
 * derivatives; they follow from Psi = sum_I c_I det A_up,I det A_dn,I (Section II) with the
 * excitation ratios t_u = det T_u of Section III: d/dc_I = t_up t_dn / S; d/dT = (1/S)
 * sum_u C_u cof(T_u); d/dPhi = A_0^{-T}[I - Tbar T^T | Tbar]; d/dB = chi^T Phibar.
 * Recomputes A_0^{-1}, T, the excitation values and S from scratch first (any pending
 * msd_ratio proposal is dropped).  The first call allocates its workspace (W x n x N and
 * W x n x n_basis doubles).  MSD_ERR_ARG if a spin's table and its adjoint do not fit in
 * one SM's shared memory. */
msd_status msd_backward(msd_ctx* ctx, const double* gbar_dev, double* dci_dev, double* dB_dev);

/* Replace the wavefunction's parameters from HOST arrays, then rebuild the state at the
 * current positions (as msd_set_positions does).  ci_host [n_det] (NULL keeps the CI
 * coefficients); B_up_host [n_basis][n_orb[0]] and B_dn_host [n_basis][n_orb[1]] (both NULL
 * keeps the orbital coefficients, both or neither).  A batched context takes ci and B
 * concatenated per system as msd_backward returns them (B_dn_host is then ignored).  Drops a
 * pending msd_ratio proposal.  Synchronises the context's stream.  With msd_backward this is
 * what a parameter optimisation needs (the paper optimises the CI coefficients in Sec. VI
 * with its own tools). */
msd_status msd_set_params(msd_ctx* ctx, const double* ci_host, const double* B_up_host, const double* B_dn_host);

/* msd_ratio without any device allocation and without keeping a proposal (the paper has no
 * counterpart: it is a library concern).  Same arguments and results as msd_ratio for the
 * current state, but the orbitals at rnew_dev go to a fixed device array of 4 MiB inside the
 * library instead of the context's proposal buffers, so a pending msd_ratio proposal stays
 * valid for msd_accept and the refresh counter does not advance.  Meant for callers that may
 * not allocate device memory when they need extra ratios (allocation can synchronise the
 * device, or the device memory is already reserved by another allocator).
 * Limits and rules: W x (5 with grad/lap, else 1) x N_spin x (8 FP64, 4 mixed) bytes must fit
 * in 4 MiB, else MSD_ERR_ARG; the array is shared by every context on a device, so calls that
 * overlap in time on one device race and must be serialised by the caller; the first call on
 * each device looks the array's address up (with that device current) and must come before
 * any stream capture the caller starts.  The context's device (current at msd_init) must be
 * the current device, else MSD_ERR_ARG.  Unlike msd_ratio it never starts the periodic
 * refresh, so after refresh_K moves of a spin it answers from the updated (not refreshed)
 * state.  Nothing is allocated or freed by this call. */
msd_status msd_ratio_noalloc(msd_ctx* ctx, int32_t elec, const double* rnew_dev, double* ratio_dev,
                             double* grad_dev, double* lap_dev);

/* Orbitals of spin `spin` at n_points positions pos_dev [n_points][3] (Algorithm 1 step 2):
 * out_dev [n_points][nch][n_orb[spin]] = phi_j and, for nch = 5, its gradient and laplacian,
 * d^a phi_j(r) = sum_mu d^a chi_mu(r) B[mu][j], in the context's orbital precision (FP64 in
 * MSD_FP64; FP32 in MSD_MIXED, where the contraction runs on the tensor cores with FP32 accuracy:
 * three TF32 pieces per operand).  The same evaluation the library runs at proposals and refreshes.
 * No state changes.  MSD_ERR_ARG for nch not 1 or 5, a batched context or the canonical method. */
msd_status msd_orbitals(msd_ctx* ctx, int32_t spin, int32_t nch, int32_t n_points, const double* pos_dev,
                        void* out_dev);

/* Walkers the FP32 path cannot represent (Section V: a reference matrix A_0 close to singular; the
 * FP32 orbitals and table then carry an error of order 2^-24 cond(A_0) or more).  At every refresh
 * of a spin the FP32 path estimates cond(A_0) = ||A_0||_inf ||A_0^{-1}||_inf per walker and spin
 * (from its FP64 inverse).  A walker whose larger estimate exceeds kappa_hold is held in an FP64
 * context of `slots` walkers: its msd_ratio, msd_accept, msd_get_state and msd_grad_lap results
 * come from there, until a later refresh finds both estimates below kappa_release.  The held set
 * changes only at refreshes (which then synchronise the stream); the FP64 context is built at
 * the first hold (an allocation).  msd_eval_batch, msd_backward and msd_ratio_noalloc use the FP32
 * state of every walker.  The FP64 work runs on an internal stream forked from and joined back into
 * the context's, overlapping the FP32 kernels of the same call.  Off by default (slots = 0); at
 * most min(W, 32) slots; suggested thresholds kappa_hold = 1e7, kappa_release = 1e5.  Releases
 * every held walker (they are held again at once if still beyond kappa_hold).  MSD_ERR_ARG for
 * other precisions, slots beyond min(W, 32) or 1 < kappa_release <= kappa_hold violated.  A
 * batched context applies it to every system. */
msd_status msd_set_rescue(msd_ctx* ctx, int32_t slots, double kappa_hold, double kappa_release);

/* out[0] = walkers held now, [1] = holds so far, [2] = releases so far, [3] = walkers beyond
 * kappa_hold that found no free slot (counted per refresh), [4] = slots; summed over systems. */
msd_status msd_rescue_stats(const msd_ctx* ctx, int64_t* out);

/* Check of the failure path of the bounded device waits (the paper has no counterpart): one kernel
 * waits on an mbarrier that nothing completes, gives up after wait_ns (1e3 .. 1e9 ns) and records
 * the timeout in the context's status word exactly as the tensor-core kernels do, so the next
 * msd_sync returns MSD_ERR_TIMEOUT (and clears it).  No GPU fault or hang is involved.
 * MSD_ERR_ARG for wait_ns outside the range or a batched context. */
msd_status msd_selftest_wait(msd_ctx* ctx, int64_t wait_ns);

/*
 * VMC energy driver.  The paper runs VMC on Psi_T = exp(J) Psi_MD (Section VI) and leaves the
 * Jastrow factor J to standard methods (Section II); these calls supply a simple one and the
 * local energy of the electronic Hamiltonian (Hartree atomic units, clamped nuclei), so a
 * Metropolis walk of Psi_T and its energy estimate run on the GPU.  Single-system contexts
 * only; everything here is FP64 in both precision modes.
 *
 * Jastrow (two-body Pade form, cusp coefficients from Kato's conditions):
 *   J = sum_{i<j} a_ij r_ij / (1 + b_ee r_ij) - sum_{i,I} Z_I r_iI / (1 + b_en r_iI),
 *   a_ij = 1/2 for electrons of unlike spin and 1/4 for like spin.
 * A parameter of 0 removes its term; msd_jastrow NULL (or both 0) means J = 0.
 */
typedef struct {
    double b_ee;  /* >= 0: electron-electron term (0 = absent) */
    double b_en;  /* >= 0: electron-nucleus term (0 = absent) */
} msd_jastrow;

/* Set the nuclear charges Z_host [n_nuc] (host, >= 0, in the order of msd_problem.nuc_xyz)
 * and the Jastrow parameters (NULL = no Jastrow).  Computes the nuclear repulsion
 * sum_{I<J} Z_I Z_J / R_IJ on the host.  May be called again to change them.  Synchronises
 * the context's stream; the first call allocates n_nuc x 32 bytes.  MSD_ERR_ARG for a
 * negative or non-finite value, or for two charged nuclei at the same point. */
msd_status msd_set_hamiltonian(msd_ctx* ctx, const double* Z_host, const msd_jastrow* jas);

/* Multiply ratio_dev [W] in place by exp(J(R') - J(R)) for the move of electron `elec` to
 * rnew_dev [W][3] from the current positions, so that msd_ratio followed by this call gives
 * Psi_T(R') / Psi_T(R) for msd_metropolis.  No state changes.  A no-op without a Jastrow term.
 * MSD_ERR_STATE before msd_set_hamiltonian or msd_set_positions. */
msd_status msd_jastrow_ratio(msd_ctx* ctx, int32_t elec, const double* rnew_dev, double* ratio_dev);

/* Local energy E_L = (H Psi_T) / Psi_T of every walker at the current positions:
 *   E_L = -1/2 sum_i lap_i Psi_T / Psi_T + sum_{i<j} 1/r_ij - sum_{i,I} Z_I / r_iI + V_nn,
 *   lap_i Psi_T / Psi_T = lap_i D / D + lap_i J + |grad_i J|^2 + 2 grad_i J . grad_i D / D,
 * with grad_i D / D and lap_i D / D of Psi_MD from the all-electron msd_grad_lap (elec = -1).
 * eloc_dev [W]; parts_dev [W][4] = (kinetic, V_ee, V_en, V_nn) or NULL.  Two particles at
 * the same point give an infinite E_L for that walker (no status is set).  The first call
 * allocates W x n_tot x 4 doubles of workspace.  MSD_ERR_STATE before msd_set_hamiltonian
 * or msd_set_positions; MSD_ERR_ARG for the canonical method. */
msd_status msd_local_energy(msd_ctx* ctx, double* eloc_dev, double* parts_dev);

/* Release every device and host resource of the context (NULL is a no-op). */
void msd_destroy(msd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MSD_H */
