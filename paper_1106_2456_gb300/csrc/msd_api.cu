// msd_api.cu -- the C ABI of libmsd (declared in include/msd.h): validation, device layout of
// the excitation strings, per-walker state and the order of kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <array>
#include <numeric>
#include <string>
#include <vector>

#include "msd.h"
#include "msd_internal.h"

using namespace msd;

namespace {

thread_local std::string g_init_error;

struct SpinConst {
    int n = 0, N = 0, m = 0, off = 0;
    void* B = nullptr;            // [nb][N] (double or float)
    float* Bsplit = nullptr;      // FP32 path: B in three TF32 pieces for the tensor-core orbitals
    TcPlan tc;
    ExcDev g;                     // device strings, grouped by order
    std::vector<int> user_of;     // internal index -> user index
    std::vector<int> internal_of; // user index -> internal index
    std::vector<long long> hist;  // strings per order 0..MAXK
    // terms grouped by this spin's internal string, used when this spin moves
    int* t_off = nullptr;         // [n_exc + 1]
    int* t_other = nullptr;       // [n_det] other spin's internal string
    double* t_c = nullptr;        // [n_det]
    int* heavy = nullptr;         // strings with many terms
    int n_heavy = 0;
    // host-side plan, uploaded by upload_spin
    std::vector<uint8_t> h_rec;
    std::vector<int> h_toff, h_tother, h_heavy;
    std::vector<double> h_tc;
    std::vector<int> h_tpos;      // term I -> its slot in the term lists of this spin (kept)
};

struct State {
    bool alloc = false, ready = false;
    double* R = nullptr;  // [W][n_tot][3]
    double* S = nullptr;  // [W] sum_u C_s[u] t_s[u] = Psi / (det A_up,0 det A_dn,0)
    double* Ainv[2] = {nullptr, nullptr};
    void* T[2] = {nullptr, nullptr};
    double* logdet[2] = {nullptr, nullptr};
    double* sgn[2] = {nullptr, nullptr};
    void* t[2] = {nullptr, nullptr};
    void* C[2] = {nullptr, nullptr};
    int since_refresh[2] = {0, 0};
    bool C_valid[2] = {false, false};
};

// Deep copy of a problem's host arrays (for building the FP64 rescue context later).
struct ProblemCopy {
    msd_problem p{};
    std::vector<double> nuc, alpha, B0, B1, ci;
    std::vector<int32_t> center, off0, off1, up, dn;
    std::vector<int8_t> lm;
    std::vector<uint8_t> h0, h1, p0, p1;
    void take(const msd_problem* q) {
        p = *q;
        nuc.assign(q->nuc_xyz, q->nuc_xyz + 3 * (size_t)q->n_nuc);
        center.assign(q->bas_center, q->bas_center + q->n_basis);
        lm.assign(q->bas_lm, q->bas_lm + q->n_basis);
        alpha.assign(q->bas_alpha, q->bas_alpha + q->n_basis);
        B0.assign(q->B[0], q->B[0] + (size_t)q->n_basis * q->n_orb[0]);
        B1.assign(q->B[1], q->B[1] + (size_t)q->n_basis * q->n_orb[1]);
        off0.assign(q->exc_off[0], q->exc_off[0] + q->n_exc[0] + 1);
        off1.assign(q->exc_off[1], q->exc_off[1] + q->n_exc[1] + 1);
        h0.assign(q->exc_holes[0], q->exc_holes[0] + off0.back());
        p0.assign(q->exc_parts[0], q->exc_parts[0] + off0.back());
        h1.assign(q->exc_holes[1], q->exc_holes[1] + off1.back());
        p1.assign(q->exc_parts[1], q->exc_parts[1] + off1.back());
        up.assign(q->det_up, q->det_up + q->n_det);
        dn.assign(q->det_dn, q->det_dn + q->n_det);
        ci.assign(q->ci, q->ci + q->n_det);
        p.nuc_xyz = nuc.data();
        p.bas_center = center.data();
        p.bas_lm = lm.data();
        p.bas_alpha = alpha.data();
        p.B[0] = B0.data();
        p.B[1] = B1.data();
        p.exc_off[0] = off0.data();
        p.exc_off[1] = off1.data();
        p.exc_holes[0] = h0.data();
        p.exc_holes[1] = h1.data();
        p.exc_parts[0] = p0.data();
        p.exc_parts[1] = p1.data();
        p.det_up = up.data();
        p.det_dn = dn.data();
        p.ci = ci.data();
    }
};

// FP32 path: walkers whose reference matrix the FP32 table cannot represent are held, from one
// refresh to a later one, in an FP64 context of a few slots (Section V: a nearly singular A_0).
struct Rescue {
    bool enabled = false;
    int slots = 0;
    double k_demote = 1e7, k_promote = 1e5;  // ||A_0||_inf ||A_0^{-1}||_inf thresholds
    msd_ctx* fb = nullptr;                   // the FP64 context (built at the first demotion)
    std::vector<int> walker_of;              // slot -> walker, -1 free
    std::vector<int> slot_of;                // walker -> slot, -1
    int active = 0;                          // slots in use (they come first in d_walker_of)
    int* d_slot_of = nullptr;                // [W]
    int* d_walker_of = nullptr;              // [slots]; free slots repeat an active walker
    int* d_status_scratch = nullptr;         // status of the FP32 kernels while some walkers are held
    double* cond[2] = {nullptr, nullptr};    // [W] per spin, from the last refresh
    double *rnew = nullptr, *ratio = nullptr, *grad = nullptr, *lap = nullptr, *R = nullptr;
    double *logabs = nullptr, *sign = nullptr, *ga_grad = nullptr, *ga_lap = nullptr;
    uint8_t* acc = nullptr;
    cudaStream_t side = nullptr;             // the FP64 context's stream, forked from the caller's
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    long long demotions = 0, promotions = 0, overflow = 0;
    int alloc_slots = 0;  // slots the scratch arrays hold
    ProblemCopy prob;
    int slots_max() const { return alloc_slots; }
};

}  // namespace

struct msd_ctx {
    int W = 0, n_tot = 0, nb = 0, K = 1;
    int device = -1;  // the CUDA device current at msd_init (whose memory holds the context)
    Rescue rs;        // FP32 path: walkers held in FP64
    bool mixed = false;
    size_t tb = 8;  // bytes of the table/orbital type
    cudaStream_t stream = nullptr;
    double4* bas = nullptr;
    float4* basf = nullptr;    // FP32 path: centres as (hi, lo) float pairs and exponents (tensor-core orbitals)
    int8_t* blm = nullptr;
    SpinConst sp[2];
    State st, scratch;
    void* Phi = nullptr;       // [W][n_max][N_max] orbitals of all electrons of one spin
    void* phi_new = nullptr;   // [W][NCH][N_max] orbitals at the proposed position
    void* phi_tmp = nullptr;   // [W][NCH][N_max] orbitals for msd_grad_lap / eval_batch
    double* rho = nullptr;     // [W]
    double* num = nullptr;     // [W][NCH]
    void* y0 = nullptr;        // [W][m_max]
    double* rnew = nullptr;    // [W][3]
    double* dummy = nullptr;   // [W] discarded ratios
    int prop_elec = -1, prop_nch = 0;
    bool prop_valid = false;
    int* d_status = nullptr;
    // staging for the host-buffer entry points
    double* d_io = nullptr;    // [W][8]
    uint8_t* d_acc = nullptr;  // [W]
    // the canonical method (MSD_CANONICAL): per spin every string's inverse and det ratio
    bool canon = false;
    double* cn_D[2] = {nullptr, nullptr};    // [W][n_exc][n][n]
    double* cn_t[2] = {nullptr, nullptr};    // [W][n_exc]
    double* cn_ru[2] = {nullptr, nullptr};   // [W][n_exc] row ratios of the proposal
    double* cn_Phi[2] = {nullptr, nullptr};  // [W][n][N] orbitals of the current positions
    uint8_t* cn_used[2] = {nullptr, nullptr};
    // all-electron gradient/laplacian workspace (allocated on first use)
    void* ga_G = nullptr;      // [W][n_max][m_max] (table precision)
    void* ga_phid = nullptr;   // [W n_max][5][N_max]
    // msd_backward: internal strings of every term, and workspace allocated on first use
    long long n_det = 0;
    int* term_iu = nullptr;    // [n_det] internal up string of term I
    int* term_id = nullptr;    // [n_det] internal down string of term I
    double* bw_M = nullptr;    // [W][n_max][N_max]
    double* bw_chi = nullptr;  // [W n_max][n_basis]
    // VMC energy driver: nuclei, charges and Jastrow (msd_set_hamiltonian), and the
    // all-electron gradient/laplacian workspace of msd_local_energy (allocated on first use)
    std::vector<double> nuc_xyz;  // [n_nuc][3] host copy
    bool ham_set = false;
    double4* ham_nuc = nullptr;   // [n_nuc] (x, y, z, Z)
    double ham_b_ee = 0.0, ham_b_en = 0.0, ham_vnn = 0.0;
    double* le_grad = nullptr;    // [W][n_tot][3]
    double* le_lap = nullptr;     // [W][n_tot]
    // batched uneven systems: one single-system context per system, run on kBatchStreams
    // internal streams forked from and joined back into `stream`
    std::vector<msd_ctx*> sub;
    std::vector<msd_ctx*> sub_parked;  // (timing: lets the batch context reuse the single-system code)
    std::vector<long long> w_off, r_off, det_off, b_off;  // per system: walkers, positions, terms, B entries
    std::vector<cudaStream_t> bstreams;
    std::vector<cudaEvent_t> bevents;                       // [0] fork, [1 + i] join of stream i
    BatchPlan bplan;                                        // single-launch descriptors of the systems
    double* b_rnew = nullptr;                               // [W][3] positions of the current proposal
    int* b_status_scratch = nullptr;                        // status word of the FP32 batched ratio launch
    // the fused step of a batch: blocks per group, chosen by timing candidate grids on the first calls
    struct StepTuning {
        std::vector<int> candidates[BatchPlan::kMaxGroups];
        int chosen[BatchPlan::kMaxGroups] = {0};
        std::vector<float> ms[BatchPlan::kMaxGroups];
        int calls = 0;
        bool done = false;
        cudaEvent_t ev[2 * BatchPlan::kMaxGroups] = {};
    } tune;
    double* step_rnew = nullptr;                            // [W][3] proposal of msd_step (single system)
    std::vector<void*> allocs;
    std::string err;
    // measurement: kernel launch count and events around the excitation-sweep kernel
    bool timing = false;
    long long launches = 0;
    long long n_refresh = 0, n_ci = 0;  // from-scratch refreshes of a spin, CI contractions (while timing)
    std::vector<cudaEvent_t> ev;  // pairs (begin, end)
    size_t ev_used = 0;
    Launch L() { return Launch{stream, d_status, timing ? &launches : nullptr}; }
    Launch L_sweep() {
        Launch l = L();
        if (timing) {
            if (ev_used + 2 > ev.size()) {
                for (int i = 0; i < 2; ++i) {
                    cudaEvent_t e = nullptr;
                    cudaEventCreate(&e);
                    ev.push_back(e);
                }
            }
            l.t0 = ev[ev_used];
            l.t1 = ev[ev_used + 1];
            ev_used += 2;
        }
        return l;
    }
};

namespace {

msd_status fail(msd_ctx* c, msd_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_init_error = buf;
    return s;
}

msd_status check_launch(msd_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return MSD_OK;
}

template <typename T>
msd_status dalloc(msd_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MSD_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return MSD_OK;
}

msd_status valloc(msd_ctx* c, void** p, size_t bytes) {
    unsigned char* q = nullptr;
    msd_status s = dalloc(c, &q, bytes);
    *p = q;
    return s;
}

template <typename T>
msd_status upload(msd_ctx* c, T** p, const T* src, size_t count) {
    msd_status s = dalloc(c, p, count);
    if (s != MSD_OK) return s;
    if (count) {
        cudaError_t e = cudaMemcpy(*p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    }
    return MSD_OK;
}

#define TRY(x)                              \
    do {                                    \
        msd_status _s = (x);                \
        if (_s != MSD_OK) return _s;        \
    } while (0)

msd_status validate(const msd_problem* p) {
    if (!p) return fail(nullptr, MSD_ERR_ARG, "problem is NULL");
    if (p->n_walkers < 1) return fail(nullptr, MSD_ERR_ARG, "n_walkers must be >= 1");
    if (p->refresh_K < 1) return fail(nullptr, MSD_ERR_ARG, "refresh_K must be >= 1");
    if (p->prec != MSD_FP64 && p->prec != MSD_MIXED && p->prec != MSD_CANONICAL)
        return fail(nullptr, MSD_ERR_ARG, "unknown precision");
    if (p->n_nuc < 1 || !p->nuc_xyz) return fail(nullptr, MSD_ERR_ARG, "need at least one nucleus");
    if (p->n_basis < 1 || !p->bas_center || !p->bas_lm || !p->bas_alpha)
        return fail(nullptr, MSD_ERR_ARG, "basis arrays missing");
    for (int mu = 0; mu < p->n_basis; ++mu) {
        if (p->bas_center[mu] < 0 || p->bas_center[mu] >= p->n_nuc)
            return fail(nullptr, MSD_ERR_ARG, "bas_center[%d] out of range", mu);
        if (p->bas_lm[mu] < 0 || p->bas_lm[mu] > 3) return fail(nullptr, MSD_ERR_ARG, "bas_lm[%d] not in 0..3", mu);
        if (!(p->bas_alpha[mu] > 0.0) || !std::isfinite(p->bas_alpha[mu]))
            return fail(nullptr, MSD_ERR_ARG, "bas_alpha[%d] must be positive and finite", mu);
    }
    for (int s = 0; s < 2; ++s) {
        const int n = p->n_elec[s], N = p->n_orb[s];
        if (n < 1 || n > MSD_MAX_ORB) return fail(nullptr, MSD_ERR_ARG, "n_elec[%d] = %d not in 1..%d", s, n, MSD_MAX_ORB);
        if (N < n || N - n > MSD_MAX_ORB) return fail(nullptr, MSD_ERR_ARG, "n_orb[%d] = %d invalid", s, N);
        if (!p->B[s]) return fail(nullptr, MSD_ERR_ARG, "B[%d] is NULL", s);
        if (p->n_exc[s] < 1 || !p->exc_off[s]) return fail(nullptr, MSD_ERR_ARG, "n_exc[%d] must be >= 1", s);
        const int32_t* off = p->exc_off[s];
        if (off[0] != 0 || off[1] != 0) return fail(nullptr, MSD_ERR_ARG, "string 0 of spin %d must be the reference", s);
        const int m = N - n;
        for (int u = 0; u < p->n_exc[s]; ++u) {
            const int k = off[u + 1] - off[u];
            if (k < 0 || k > MSD_MAX_ORDER || k > n || k > m)
                return fail(nullptr, MSD_ERR_ARG, "string %d of spin %d has invalid order %d", u, s, k);
            if (k && (!p->exc_holes[s] || !p->exc_parts[s]))
                return fail(nullptr, MSD_ERR_ARG, "hole/particle arrays of spin %d missing", s);
            for (int q = 0; q < k; ++q) {
                const int h = p->exc_holes[s][off[u] + q], pa = p->exc_parts[s][off[u] + q];
                if (h >= n || pa >= m)
                    return fail(nullptr, MSD_ERR_ARG, "string %d of spin %d: index out of range", u, s);
                if (q && (h <= p->exc_holes[s][off[u] + q - 1] || pa <= p->exc_parts[s][off[u] + q - 1]))
                    return fail(nullptr, MSD_ERR_ARG, "string %d of spin %d: indices not strictly ascending", u, s);
            }
        }
    }
    if (p->n_det < 1 || !p->det_up || !p->det_dn || !p->ci) return fail(nullptr, MSD_ERR_ARG, "term arrays missing");
    if (p->n_det > (int64_t)0x7fffffff) return fail(nullptr, MSD_ERR_ARG, "n_det too large");
    for (int64_t I = 0; I < p->n_det; ++I) {
        if (p->det_up[I] < 0 || p->det_up[I] >= p->n_exc[0] || p->det_dn[I] < 0 || p->det_dn[I] >= p->n_exc[1])
            return fail(nullptr, MSD_ERR_ARG, "term %lld refers to a missing string", (long long)I);
        if (!std::isfinite(p->ci[I])) return fail(nullptr, MSD_ERR_ARG, "ci[%lld] not finite", (long long)I);
    }
    const bool mixed = p->prec == MSD_MIXED;
    for (int s = 0; s < 2; ++s) {
        const int n = p->n_elec[s], m = p->n_orb[s] - p->n_elec[s];
        const size_t need = ratio_smem_bytes(mixed, n, m, NCH);
        const size_t inv = (size_t)n * (n + 1) * 8 + (size_t)n * 12 + 16;
        // (also bounds n below 255, so hole byte 0xFF can mark an empty record slot)
        if (need > 220 * 1024 || inv > 220 * 1024 || n >= (int)kEmptyRecord)
            return fail(nullptr, MSD_ERR_ARG,
                        "spin %d: per-walker table (%d x %d) does not fit in one SM's shared memory", s, n, m);
    }
    return MSD_OK;
}

// Build device strings of spin s, grouped by order and sorted within each order.  Singles
// become a dense n x m block of internal indices when at least a quarter of them are present.
// Packs the strings of order k into warp batches of kBatch internal slots (Section III
// excitations, one per lane of a warp).  Within a batch the particle in slot l of every
// excitation has a distinct residue mod 32, so the lanes' scatter-adds into G never collide and
// their table reads T[h][p] (row stride a multiple of 32) fall in distinct shared-memory banks.
// The particles of an excitation may sit in any slot order; its holes are permuted with the same
// parity, which leaves det T_u and the per-particle entries of adj(T_u) x_u unchanged.  Each
// string goes to the first of the kWindow most recently opened batches where a slot assignment
// exists (a bipartite matching of its particles to free slots), else opens a new batch; unused
// slots hold kEmptyRecord records.
// Without `conflict_free` (FP64 tables, whose sweep is bound by FP64 arithmetic rather than by
// shared-memory banks) the strings fill the batches in their sorted order.
// Returns the number of internal slots used (a multiple of kBatch).
int pack_group(SpinConst& S, const msd_problem* p, int s, int k, const int* members, int count, int idx0,
               std::vector<uint8_t>& rec, bool conflict_free) {
    constexpr int kWindow = 512;
    const int32_t* off = p->exc_off[s];
    struct Batch {
        uint32_t used[MAXK];
        int cnt;
    };
    std::vector<Batch> batches;
    std::vector<int> batch_of(count), lane_of(count);
    std::vector<std::array<int8_t, MAXK>> slot_of(count);
    int first_open = 0;
    int res[MAXK], owner[MAXK], slot[MAXK];
    // augmenting-path search: particle i takes a slot whose residue bit is free
    std::function<bool(const Batch&, int, unsigned&)> augment = [&](const Batch& b, int i, unsigned& seen) {
        for (int l = 0; l < k; ++l) {
            if (((b.used[l] >> res[i]) & 1u) || ((seen >> l) & 1u)) continue;
            seen |= 1u << l;
            if (owner[l] < 0 || augment(b, owner[l], seen)) {
                owner[l] = i;
                slot[i] = l;
                return true;
            }
        }
        return false;
    };
    auto fits = [&](const Batch& b) {
        for (int l = 0; l < k; ++l) owner[l] = -1;
        for (int i = 0; i < k; ++i) {
            unsigned seen = 0;
            if (!augment(b, i, seen)) return false;
        }
        return true;
    };
    for (int e = 0; e < count; ++e) {
        const int u = members[e];
        for (int i = 0; i < k; ++i) res[i] = p->exc_parts[s][off[u] + i] & 31;
        int bi = -1;
        const int last = (int)batches.size();
        if (!conflict_free) {
            if (last > 0 && batches[last - 1].cnt < kBatch) bi = last - 1;
            for (int i = 0; i < k; ++i) slot[i] = i;
        } else {
            for (int b = std::max(first_open, last - kWindow); b < last && bi < 0; ++b)
                if (batches[b].cnt < kBatch && fits(batches[b])) bi = b;
        }
        if (bi < 0) {
            batches.push_back(Batch{});
            bi = (int)batches.size() - 1;
            for (int i = 0; i < k; ++i) slot[i] = i;
        }
        Batch& b = batches[bi];
        for (int i = 0; i < k; ++i) {
            b.used[slot[i]] |= 1u << res[i];
            slot_of[e][i] = (int8_t)slot[i];
        }
        batch_of[e] = bi;
        lane_of[e] = b.cnt++;
        while (first_open < (int)batches.size() && batches[first_open].cnt == kBatch) ++first_open;
    }
    const int rb = rec_bytes(k);
    const size_t base = rec.size();
    rec.resize(base + (size_t)batches.size() * kBatch * rb, kEmptyRecord);
    for (int e = 0; e < count; ++e) {
        const int u = members[e];
        const int i_int = batch_of[e] * kBatch + lane_of[e];
        S.internal_of[u] = idx0 + i_int;
        uint8_t* r = rec.data() + base + (size_t)i_int * rb;
        for (int q = 0; q < rb; ++q) r[q] = 0;
        int inv = 0;  // parity of the particle placement
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j) inv += slot_of[e][i] > slot_of[e][j];
        for (int q = 0; q < k; ++q) r[q] = p->exc_holes[s][off[u] + q];
        if (inv & 1) std::swap(r[0], r[1]);  // odd placement (k >= 2): an odd hole permutation
        for (int i = 0; i < k; ++i) r[k + slot_of[e][i]] = p->exc_parts[s][off[u] + i];
    }
    return (int)batches.size() * kBatch;
}

msd_status plan_strings(SpinConst& S, const msd_problem* p, int s) {
    const int ne = p->n_exc[s];
    const int32_t* off = p->exc_off[s];
    auto order_of = [&](int u) { return off[u + 1] - off[u]; };
    S.hist.assign(MAXK + 1, 0);
    S.g.kmax = 0;
    for (int u = 0; u < ne; ++u) {
        S.hist[order_of(u)]++;
        S.g.kmax = std::max(S.g.kmax, order_of(u));
    }
    const bool dense1 = S.hist[1] > 0 && 4 * S.hist[1] >= (long long)S.n * S.m;
    S.g.dense1 = dense1 ? 1 : 0;
    std::vector<int> order(ne);
    std::iota(order.begin(), order.end(), 0);
    auto key_less = [&](int a, int b) {
        const int ka = order_of(a), kb = order_of(b);
        if (ka != kb) return ka < kb;
        for (int q = 0; q < ka; ++q) {
            const int ha = p->exc_holes[s][off[a] + q], hb = p->exc_holes[s][off[b] + q];
            if (ha != hb) return ha < hb;
        }
        for (int q = 0; q < ka; ++q) {
            const int pa = p->exc_parts[s][off[a] + q], pb = p->exc_parts[s][off[b] + q];
            if (pa != pb) return pa < pb;
        }
        return a < b;
    };
    std::stable_sort(order.begin(), order.end(), key_less);  // the reference (k = 0, index 0) stays first
    S.internal_of.assign(ne, -1);
    std::vector<uint8_t> rec;
    for (int k = 0; k <= MAXK + 1; ++k) S.g.roff[k] = 0;
    int idx = 0, pos = 0;
    for (int k = 0; k <= MAXK; ++k) {
        S.g.goff[k] = idx;
        while (rec.size() % 16) rec.push_back(0);
        S.g.roff[k] = (long long)rec.size();
        const int first = pos;
        while (pos < ne && order_of(order[pos]) == k) ++pos;
        if (k == 0) {
            for (int i = first; i < pos; ++i) S.internal_of[order[i]] = idx++;
        } else if (k == 1 && dense1) {
            for (int i = first; i < pos; ++i) {
                const int u = order[i];
                S.internal_of[u] = idx + p->exc_holes[s][off[u]] * S.m + p->exc_parts[s][off[u]];
            }
            idx += S.n * S.m;
        } else if (pos > first) {
            idx += pack_group(S, p, s, k, order.data() + first, pos - first, idx, rec, p->prec == MSD_MIXED);
        }
    }
    while (rec.size() % 16) rec.push_back(0);
    S.g.goff[MAXK + 1] = idx;
    S.g.n_exc = idx;
    S.user_of.assign(idx, -1);
    for (int u = 0; u < ne; ++u) S.user_of[S.internal_of[u]] = u;
    S.h_rec.swap(rec);
    S.g.rec = nullptr;
    return MSD_OK;
}

// Terms grouped by the internal string of spin s (the moving spin), for C_s.
msd_status plan_terms(SpinConst& S, const SpinConst& O, const msd_problem* p, int s) {
    const int ne = S.g.n_exc;  // internal strings (a dense singles block counts n m)
    const int64_t nd = p->n_det;
    const int32_t* mine = s == 0 ? p->det_up : p->det_dn;
    const int32_t* oth = s == 0 ? p->det_dn : p->det_up;
    std::vector<int> off(ne + 1, 0);
    for (int64_t I = 0; I < nd; ++I) off[S.internal_of[mine[I]] + 1]++;
    for (int u = 0; u < ne; ++u) off[u + 1] += off[u];
    std::vector<int> pos(off.begin(), off.end() - 1);
    std::vector<int> other(nd);
    std::vector<double> cc(nd);
    S.h_tpos.assign(nd, 0);
    for (int64_t I = 0; I < nd; ++I) {
        const int u = S.internal_of[mine[I]];
        const int q = pos[u]++;
        other[q] = O.internal_of[oth[I]];
        cc[q] = p->ci[I];
        S.h_tpos[I] = q;
    }
    std::vector<int> heavy;
    for (int u = 0; u < ne; ++u)
        if (off[u + 1] - off[u] > heavy_threshold()) heavy.push_back(u);
    S.h_toff.swap(off);
    S.h_tother.swap(other);
    S.h_tc.swap(cc);
    S.h_heavy.swap(heavy);
    S.n_heavy = (int)S.h_heavy.size();
    return MSD_OK;
}

// Host plan of both spins: validation already done; no CUDA call.
msd_status plan_problem(SpinConst (&sp)[2], const msd_problem* p) {
    for (int s = 0; s < 2; ++s) {
        sp[s].n = p->n_elec[s];
        sp[s].N = p->n_orb[s];
        sp[s].m = p->n_orb[s] - p->n_elec[s];
        sp[s].off = s ? p->n_elec[0] : 0;
        TRY(plan_strings(sp[s], p, s));
    }
    for (int s = 0; s < 2; ++s) TRY(plan_terms(sp[s], sp[1 - s], p, s));
    return MSD_OK;
}

msd_status upload_spin(msd_ctx* c, SpinConst& S) {
    uint8_t* d_rec = nullptr;
    TRY(upload(c, &d_rec, S.h_rec.data(), S.h_rec.size()));
    S.g.rec = d_rec;
    TRY(upload(c, &S.t_off, S.h_toff.data(), S.h_toff.size()));
    TRY(upload(c, &S.t_other, S.h_tother.data(), S.h_tother.size()));
    TRY(upload(c, &S.t_c, S.h_tc.data(), S.h_tc.size()));
    TRY(upload(c, &S.heavy, S.h_heavy.data(), S.h_heavy.size()));
    std::vector<uint8_t>().swap(S.h_rec);
    std::vector<int>().swap(S.h_toff);
    std::vector<int>().swap(S.h_tother);
    std::vector<double>().swap(S.h_tc);
    std::vector<int>().swap(S.h_heavy);
    return MSD_OK;
}

msd_status alloc_state(msd_ctx* c, State& st) {
    if (st.alloc) return MSD_OK;
    const size_t W = c->W;
    TRY(dalloc(c, &st.R, W * c->n_tot * 3));
    TRY(dalloc(c, &st.S, W));
    for (int s = 0; s < 2; ++s) {
        const SpinConst& S = c->sp[s];
        TRY(dalloc(c, &st.Ainv[s], W * S.n * S.n));
        TRY(valloc(c, &st.T[s], W * S.n * std::max(S.m, 1) * c->tb));
        TRY(dalloc(c, &st.logdet[s], W));
        TRY(dalloc(c, &st.sgn[s], W));
        TRY(valloc(c, &st.t[s], W * S.g.n_exc * c->tb));
        TRY(valloc(c, &st.C[s], W * S.g.n_exc * c->tb));
    }
    st.alloc = true;
    return MSD_OK;
}

// Orbitals of spin s at P points (Algorithm 1 step 2): on the tensor cores for the FP32 path,
// by the SIMT product in FP64.
void orbitals(msd_ctx* c, const SpinConst& S, int nch, int P, int ppw, const double* pos, long long wstride,
              int p_off, void* out) {
    if (c->mixed && S.Bsplit)
        launch_orbitals_tc(c->L(), nch, P, ppw, pos, wstride, p_off, c->basf, c->blm, c->nb, S.tc, S.Bsplit, S.N,
                           static_cast<float*>(out));
    else
        launch_orbitals(c->L(), c->mixed, nch, P, ppw, pos, wstride, p_off, c->bas, c->blm, c->nb, S.B, S.N, out);
}

// The three TF32 pieces of B_s (from its FP64 value) for the tensor-core orbitals.
msd_status upload_split_B(msd_ctx* c, SpinConst& S, const double* B_host) {
    std::vector<float> h(S.tc.floats);
    tc_split_B(S.tc, c->nb, S.N, B_host, h.data());
    if (!S.Bsplit) TRY(dalloc(c, &S.Bsplit, h.size()));
    const cudaError_t e = cudaMemcpy(S.Bsplit, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "upload of the split B: %s", cudaGetErrorString(e));
    return MSD_OK;
}

// A7: recompute A_0^{-1}, log|det A_0| and T of spin s from the positions (Section III).
msd_status refresh_spin(msd_ctx* c, State& st, int s) {
    const SpinConst& S = c->sp[s];
    orbitals(c, S, 1, c->W * S.n, S.n, st.R, (long long)c->n_tot * 3, S.off, c->Phi);
    launch_inverse(c->L(), c->mixed, c->W, S.n, S.N, c->Phi, st.Ainv[s], st.logdet[s], st.sgn[s],
                   (c->rs.enabled && &st == &c->st) ? c->rs.cond[s] : nullptr);
    if (S.m > 0) {
        if (c->mixed && table_tc_supported(S.n))
            launch_table_tc(c->L(), c->W, S.n, S.N, st.Ainv[s], static_cast<const float*>(c->Phi),
                            static_cast<float*>(st.T[s]));
        else
            launch_table(c->L(), c->mixed, c->W, S.n, S.N, st.Ainv[s], c->Phi, st.T[s]);
    }
    if (c->timing) c->n_refresh++;
    st.since_refresh[s] = 0;
    st.C_valid[1 - s] = false;  // C of the other spin depends on this spin's t
    return check_launch(c, "refresh");
}

// C_s from the current table of the other spin.
msd_status ensure_C(msd_ctx* c, State& st, int s) {
    if (st.C_valid[s]) return MSD_OK;
    const SpinConst& S = c->sp[s];
    const SpinConst& O = c->sp[1 - s];
    launch_exc_det(c->L(), c->mixed, c->W, O.n, O.m, O.g, st.T[1 - s], st.t[1 - s]);
    launch_ci_contract(c->L(), c->mixed, c->W, S.g.n_exc, O.g.n_exc, S.t_off, S.t_other, S.t_c, st.t[1 - s], st.C[s]);
    launch_ci_contract_heavy(c->L(), c->mixed, c->W, S.g.n_exc, O.g.n_exc, S.n_heavy, S.heavy, S.t_off, S.t_other,
                             S.t_c, st.t[1 - s], st.C[s]);
    if (c->timing) c->n_ci++;
    st.C_valid[s] = true;
    return check_launch(c, "CI contraction");
}

// S = sum_u C_s[u] t_s[u] from the current table of spin s.
msd_status recompute_S(msd_ctx* c, State& st, int s) {
    const SpinConst& S = c->sp[s];
    launch_exc_det(c->L(), c->mixed, c->W, S.n, S.m, S.g, st.T[s], st.t[s]);
    launch_ci_dot(c->L(), c->mixed, c->W, S.g.n_exc, st.C[s], st.t[s], st.S);
    return check_launch(c, "CI sum");
}

msd_status rebuild(msd_ctx* c, State& st);

msd_status set_positions(msd_ctx* c, State& st, const double* R_dev) {
    cudaError_t e = cudaMemcpyAsync(st.R, R_dev, sizeof(double) * c->W * c->n_tot * 3, cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "copy of positions: %s", cudaGetErrorString(e));
    return rebuild(c, st);
}

// Everything from scratch at the positions in st.R (Section III: A_0^{-1} and every
// determinant recomputed directly rather than updated).
msd_status canon_refresh(msd_ctx* c, State& st, int s);
msd_status canon_C(msd_ctx* c, State& st, int s, bool with_S);

msd_status rebuild(msd_ctx* c, State& st) {
    if (c->canon) {
        TRY(canon_refresh(c, st, 0));
        TRY(canon_refresh(c, st, 1));
        st.C_valid[0] = st.C_valid[1] = false;
        TRY(canon_C(c, st, 0, true));
        st.ready = true;
        return MSD_OK;
    }
    TRY(refresh_spin(c, st, 0));
    TRY(refresh_spin(c, st, 1));
    st.C_valid[0] = st.C_valid[1] = false;
    TRY(ensure_C(c, st, 0));
    TRY(recompute_S(c, st, 0));
    st.ready = true;
    return MSD_OK;
}

// The canonical method: every string's inverse and det ratio of spin s from scratch at the
// positions in st.R (orbitals of all the spin's electrons, the reference inverse for det A_0).
msd_status canon_refresh(msd_ctx* c, State& st, int s) {
    const SpinConst& S = c->sp[s];
    launch_orbitals(c->L(), false, 1, c->W * S.n, S.n, st.R, (long long)c->n_tot * 3, S.off, c->bas, c->blm, c->nb,
                    S.B, S.N, c->cn_Phi[s]);
    launch_inverse(c->L(), false, c->W, S.n, S.N, c->cn_Phi[s], st.Ainv[s], st.logdet[s], st.sgn[s]);
    launch_canon_build(c->L(), c->W, S.n, S.N, S.m, S.g, c->cn_Phi[s], c->cn_used[s], st.logdet[s], st.sgn[s],
                       c->cn_D[s], c->cn_t[s]);
    st.since_refresh[s] = 0;
    st.C_valid[1 - s] = false;
    return check_launch(c, "canonical refresh");
}

// C_s from the other spin's det ratios, then S = sum_u C_s[u] t_s[u].
msd_status canon_C(msd_ctx* c, State& st, int s, bool with_S) {
    const SpinConst& S = c->sp[s];
    const SpinConst& O = c->sp[1 - s];
    if (!st.C_valid[s]) {
        launch_ci_contract(c->L(), false, c->W, S.g.n_exc, O.g.n_exc, S.t_off, S.t_other, S.t_c, c->cn_t[1 - s], st.C[s]);
        launch_ci_contract_heavy(c->L(), false, c->W, S.g.n_exc, O.g.n_exc, S.n_heavy, S.heavy, S.t_off, S.t_other,
                                 S.t_c, c->cn_t[1 - s], st.C[s]);
        st.C_valid[s] = true;
    }
    if (with_S) launch_ci_dot(c->L(), false, c->W, S.g.n_exc, st.C[s], c->cn_t[s], st.S);
    return check_launch(c, "canonical CI sums");
}

int spin_of(const msd_ctx* c, int e) { return e < c->sp[0].n ? 0 : 1; }

// ------------------------------------------------------------------------------------------
// FP64 rescue of ill-conditioned walkers on the FP32 path
// ------------------------------------------------------------------------------------------
bool rescue_on(const msd_ctx* c) { return c->rs.enabled && c->rs.active > 0; }

// Per-walker arrays of a mixed single-system context; slots = min(W, 32).
msd_status rescue_alloc(msd_ctx* c, const msd_problem* p) {
    Rescue& r = c->rs;
    r.enabled = c->mixed;
    if (!r.enabled) return MSD_OK;
    r.slots = 0;  // off until msd_set_rescue
    r.alloc_slots = std::min(c->W, 32);
    r.walker_of.assign(r.alloc_slots, -1);
    r.slot_of.assign(c->W, -1);
    const size_t W = c->W, S = r.alloc_slots, nt = c->n_tot;
    TRY(dalloc(c, &r.cond[0], W));
    TRY(dalloc(c, &r.cond[1], W));
    TRY(dalloc(c, &r.d_slot_of, W));
    TRY(dalloc(c, &r.d_walker_of, S));
    TRY(dalloc(c, &r.d_status_scratch, 1));
    TRY(dalloc(c, &r.rnew, S * 3));
    TRY(dalloc(c, &r.ratio, S));
    TRY(dalloc(c, &r.grad, S * 3));
    TRY(dalloc(c, &r.lap, S));
    TRY(dalloc(c, &r.R, S * nt * 3));
    TRY(dalloc(c, &r.logabs, S));
    TRY(dalloc(c, &r.sign, S));
    TRY(dalloc(c, &r.acc, S));
    TRY(dalloc(c, &r.ga_grad, S * nt * 3));
    TRY(dalloc(c, &r.ga_lap, S * nt));
    if (cudaMemset(r.cond[0], 0, sizeof(double) * W) != cudaSuccess ||
        cudaMemset(r.cond[1], 0, sizeof(double) * W) != cudaSuccess ||
        cudaMemset(r.d_slot_of, 0xFF, sizeof(int) * W) != cudaSuccess)
        return fail(c, MSD_ERR_CUDA, "rescue memset");
    r.prob.take(p);
    return MSD_OK;
}

msd_status rescue_upload_maps(msd_ctx* c) {
    Rescue& r = c->rs;
    std::vector<int> wo(r.slots);
    for (int q = 0; q < r.slots; ++q) wo[q] = q < r.active ? r.walker_of[q] : (r.active ? r.walker_of[0] : 0);
    cudaError_t e = cudaMemcpyAsync(r.d_walker_of, wo.data(), sizeof(int) * r.slots, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r.d_slot_of, r.slot_of.data(), sizeof(int) * c->W, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host vectors may change before the copy ran
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "rescue maps: %s", cudaGetErrorString(e));
    return MSD_OK;
}

// Release every held walker (new positions).
msd_status rescue_reset(msd_ctx* c) {
    Rescue& r = c->rs;
    if (!r.enabled) return MSD_OK;
    std::fill(r.walker_of.begin(), r.walker_of.end(), -1);
    std::fill(r.slot_of.begin(), r.slot_of.end(), -1);
    r.active = 0;
    return rescue_upload_maps(c);
}

// The FP64 context runs on its own stream, forked from and joined back into the caller's, so its
// work overlaps the FP32 kernels of the same call.
msd_status side_fork(msd_ctx* c) {
    Rescue& r = c->rs;
    cudaError_t e = cudaEventRecord(r.ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(r.side, r.ev_fork, 0);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "rescue fork: %s", cudaGetErrorString(e));
    return MSD_OK;
}

msd_status side_join(msd_ctx* c) {
    Rescue& r = c->rs;
    cudaError_t e = cudaEventRecord(r.ev_join, r.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, r.ev_join, 0);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "rescue join: %s", cudaGetErrorString(e));
    return MSD_OK;
}

Launch side_launch(msd_ctx* c) {
    Launch l = c->L();
    l.stream = c->rs.side;
    return l;
}

// After a refresh of the main state: hold walkers whose condition estimate (the larger of the two
// spins' latest) exceeds k_demote, release held ones below k_promote, and rebuild the FP64
// context at the held walkers' current positions when the set changed.  Synchronises the stream.
msd_status rescue_update(msd_ctx* c) {
    Rescue& r = c->rs;
    if (!r.enabled || r.slots == 0) return MSD_OK;
    const size_t W = c->W;
    std::vector<double> k0(W), k1(W);
    cudaError_t e = cudaMemcpyAsync(k0.data(), r.cond[0], sizeof(double) * W, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(k1.data(), r.cond[1], sizeof(double) * W, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "rescue read: %s", cudaGetErrorString(e));
    bool changed = false;
    for (size_t w = 0; w < W; ++w) {
        const double k = std::max(k0[w], k1[w]);
        const int q = r.slot_of[w];
        if (q < 0 && !(k <= r.k_demote)) {  // also a non-finite estimate
            int free = -1;
            for (int j = 0; j < r.slots && free < 0; ++j)
                if (r.walker_of[j] < 0) free = j;
            if (free < 0) {
                ++r.overflow;
                continue;
            }
            r.walker_of[free] = (int)w;
            r.slot_of[w] = free;
            ++r.demotions;
            changed = true;
        } else if (q >= 0 && k < r.k_promote) {
            r.walker_of[q] = -1;
            r.slot_of[w] = -1;
            ++r.promotions;
            changed = true;
        }
    }
    if (!changed) return MSD_OK;
    // held walkers first, in slot order
    std::vector<int> held;
    for (int j = 0; j < r.slots; ++j)
        if (r.walker_of[j] >= 0) held.push_back(r.walker_of[j]);
    r.active = (int)held.size();
    std::fill(r.walker_of.begin(), r.walker_of.end(), -1);
    std::fill(r.slot_of.begin(), r.slot_of.end(), -1);
    for (int j = 0; j < r.active; ++j) {
        r.walker_of[j] = held[j];
        r.slot_of[held[j]] = j;
    }
    TRY(rescue_upload_maps(c));
    if (r.active == 0) return MSD_OK;
    if (!r.side) {
        if (cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.ev_join, cudaEventDisableTiming) != cudaSuccess)
            return fail(c, MSD_ERR_CUDA, "rescue stream");
    }
    if (!r.fb) {
        msd_problem q = r.prob.p;
        q.prec = MSD_FP64;
        q.n_walkers = r.slots;
        q.refresh_K = c->K;
        q.cuda_stream = r.side;
        const msd_status st = msd_init(&q, 1, &r.fb);
        if (st != MSD_OK) return fail(c, st, "FP64 rescue context: %s", msd_last_error(nullptr));
    }
    TRY(side_fork(c));
    launch_gather_rows(side_launch(c), r.slots, r.d_walker_of, c->n_tot * 3, c->st.R, r.R);
    const msd_status st = msd_set_positions(r.fb, r.R);
    if (st != MSD_OK) return fail(c, st, "FP64 rescue: %s", r.fb->err.c_str());
    TRY(side_join(c));
    return check_launch(c, "rescue rebuild");
}

msd_status rescue_fail(msd_ctx* c, msd_status st) {
    return fail(c, st, "FP64 rescue: %s", c->rs.fb ? c->rs.fb->err.c_str() : "");
}

// The held walkers' ratio (and gradient, laplacian) from the FP64 context: started on its stream
// before the FP32 sweep, written over the FP32 values after it, then the finiteness check the
// FP32 launch was relieved of.
msd_status rescue_ratio_begin(msd_ctx* c, int elec, const double* rnew_dev, bool with_grad) {
    Rescue& r = c->rs;
    TRY(side_fork(c));
    launch_gather_rows(side_launch(c), r.slots, r.d_walker_of, 3, rnew_dev, r.rnew);
    const msd_status st = msd_ratio(r.fb, elec, r.rnew, r.ratio, with_grad ? r.grad : nullptr,
                                    with_grad ? r.lap : nullptr);
    if (st != MSD_OK) return rescue_fail(c, st);
    return MSD_OK;
}

msd_status rescue_ratio_end(msd_ctx* c, double* ratio, double* grad, double* lap) {
    Rescue& r = c->rs;
    TRY(side_join(c));
    launch_scatter_rows(c->L(), r.active, r.d_walker_of, 1, r.ratio, ratio);
    if (grad) {
        launch_scatter_rows(c->L(), r.active, r.d_walker_of, 3, r.grad, grad);
        launch_scatter_rows(c->L(), r.active, r.d_walker_of, 1, r.lap, lap);
    }
    launch_check_finite(c->L(), c->W, ratio);
    return check_launch(c, "rescue ratio");
}

msd_status rescue_ratio(msd_ctx* c, int elec, const double* rnew_dev, double* ratio, double* grad, double* lap) {
    TRY(rescue_ratio_begin(c, elec, rnew_dev, grad != nullptr));
    return rescue_ratio_end(c, ratio, grad, lap);
}

// The held walkers' accept on the FP64 stream, overlapping the FP32 accept.
msd_status rescue_accept_begin(msd_ctx* c, int elec, const uint8_t* accept_dev) {
    Rescue& r = c->rs;
    TRY(side_fork(c));
    launch_gather_bytes(side_launch(c), r.slots, r.d_walker_of, accept_dev, r.acc);
    const msd_status st = msd_accept(r.fb, elec, r.acc);
    if (st != MSD_OK) return rescue_fail(c, st);
    return MSD_OK;
}

msd_status rescue_accept(msd_ctx* c, int elec, const uint8_t* accept_dev) {
    TRY(rescue_accept_begin(c, elec, accept_dev));
    TRY(side_join(c));
    return check_launch(c, "rescue accept");
}

// Orbitals at the current position of electron e, then the bordered sweep with rnew = r_e.
msd_status grad_lap_one(msd_ctx* c, State& st, int e, double* grad, long long gs, double* lap, long long ls) {
    const int s = spin_of(c, e);
    const SpinConst& S = c->sp[s];
    TRY(ensure_C(c, st, s));
    orbitals(c, S, NCH, c->W, 1, st.R, (long long)c->n_tot * 3, e, c->phi_tmp);
    RatioArgs a{};
    a.W = c->W; a.n = S.n; a.N = S.N; a.m = S.m; a.row = e - S.off; a.nch = NCH;
    a.phi = c->phi_tmp; a.Ainv = st.Ainv[s]; a.T = st.T[s]; a.C = st.C[s]; a.S = st.S; a.g = S.g;
    a.ratio = c->dummy; a.rs = 1; a.grad = grad; a.gs = gs; a.lap = lap; a.ls = ls;
    if (S.m == 0) a.g.kmax = 0;
    launch_ratio(c->L_sweep(), c->mixed, a);
    return check_launch(c, "grad/lap");
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

constexpr int kBatchStreams = 8;

bool is_batch(const msd_ctx* c) { return c && !c->sub.empty(); }

// Make every internal stream wait for the work queued so far on the caller's stream.
msd_status batch_fork(msd_ctx* c) {
    cudaError_t e = cudaEventRecord(c->bevents[0], c->stream);
    for (size_t i = 0; e == cudaSuccess && i < c->bstreams.size(); ++i)
        e = cudaStreamWaitEvent(c->bstreams[i], c->bevents[0], 0);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "fork: %s", cudaGetErrorString(e));
    return MSD_OK;
}

// Make the caller's stream wait for everything queued on the internal streams.
msd_status batch_join(msd_ctx* c) {
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; e == cudaSuccess && i < c->bstreams.size(); ++i) {
        e = cudaEventRecord(c->bevents[1 + i], c->bstreams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->bevents[1 + i], 0);
    }
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "join: %s", cudaGetErrorString(e));
    return MSD_OK;
}

// Run f(system index, sub-context) for every system between a fork and a join; the first
// failure is reported with the system's index.
template <typename F>
msd_status batch_each(msd_ctx* c, F&& f) {
    TRY(batch_fork(c));
    for (size_t s = 0; s < c->sub.size(); ++s) {
        const msd_status st = f((int)s, c->sub[s]);
        if (st != MSD_OK) {
            batch_join(c);
            return fail(c, st, "system %zu: %s", s, c->sub[s]->err.c_str());
        }
    }
    return batch_join(c);
}

int sub_elec(const msd_ctx* c, int s, int elec) { return elec % c->sub[s]->n_tot; }

// Descriptors of every system for the single-launch stages (orbitals at r', ratio, accept,
// proposal): pointers into each system's own context, per spin.
msd_status build_batch_plan(msd_ctx* c) {
    const int ns = (int)c->sub.size();
    std::vector<BatchSys> sys(ns);
    std::vector<int4> tiles, tc_tiles;
    std::vector<int> wsys;
    size_t tc_smem = 0;
    std::vector<size_t> sys_smem(ns, 0);
    size_t rsm = 0, asm_ = 0;
    const int TP = orbital_tile_points(), TJ = orbital_tile_orbitals();
    for (int q = 0; q < ns; ++q) {
        msd_ctx* sc = c->sub[q];
        BatchSys& B = sys[q];
        B.n_tot = sc->n_tot;
        B.n_up = sc->sp[0].n;
        B.W = sc->W;
        B.w_off = (int)c->w_off[q];
        B.status = sc->d_status;
        // FP32 path: the ratio launch reports into a scratch word; the outputs are checked after the
        // held walkers' FP64 values replaced theirs
        B.ratio_status = c->mixed ? c->b_status_scratch : nullptr;
        B.R = sc->st.R;
        int Nmax = 0, nT = 0;
        for (int s = 0; s < 2; ++s) {
            const SpinConst& S = sc->sp[s];
            B.orb[s] = OrbArgs{sc->bas, sc->blm, sc->nb, S.B, S.N, sc->phi_new, S.Bsplit, S.tc.TN, S.tc.nT, sc->basf};
            if (S.Bsplit) tc_smem = std::max(tc_smem, S.tc.smem);
            nT = std::max(nT, S.tc.nT);
            RatioArgs& a = B.ratio[s];
            a = RatioArgs{};
            a.W = sc->W; a.n = S.n; a.N = S.N; a.m = S.m;
            a.phi = sc->phi_new; a.Ainv = sc->st.Ainv[s]; a.T = sc->st.T[s]; a.C = sc->st.C[s]; a.S = sc->st.S;
            a.g = S.g;
            if (S.m == 0) a.g.kmax = 0;
            a.rho = sc->rho; a.num = sc->num; a.y0 = sc->y0;
            AcceptArgs& b = B.accept[s];
            b = AcceptArgs{};
            b.W = sc->W; b.n = S.n; b.N = S.N; b.m = S.m; b.n_tot = sc->n_tot;
            b.phi = sc->phi_new; b.rho = sc->rho; b.num = sc->num; b.y0 = sc->y0;
            b.Ainv = sc->st.Ainv[s]; b.T = sc->st.T[s]; b.R = sc->st.R; b.logdet = sc->st.logdet[s];
            b.sgn = sc->st.sgn[s]; b.S = sc->st.S;
            b.skip = sc->rs.d_slot_of;
            sys_smem[q] = std::max(sys_smem[q], ratio_smem_bytes(c->mixed, S.n, S.m, NCH));
            rsm = std::max(rsm, sys_smem[q]);
            asm_ = std::max(asm_, accept_smem_bytes(S.n));
            Nmax = std::max(Nmax, S.N);
        }
        for (int w = 0; w < sc->W; ++w) wsys.push_back(q);
        for (int p0 = 0; p0 < sc->W; p0 += TP)
            for (int j0 = 0; j0 < Nmax; j0 += TJ) tiles.push_back(make_int4(q, p0, j0, 0));
        if (c->mixed) {
            const int ppt = tc_tile_points(NCH);  // the five-channel tiling covers the one-channel one
            for (int x = 0; x * ppt < sc->W; ++x)
                for (int y = 0; y < nT; ++y) tc_tiles.push_back(make_int4(q, x, y, 0));
        }
    }
    // ratio blocks grouped by shared-memory size class (the CTAs an SM can hold), largest last
    auto cls = [&](size_t sm) {
        const size_t per_sm = 227 * 1024;
        const int fit = (int)std::min<size_t>(3, per_sm / (sm + 1024));
        return fit >= 3 ? 0 : fit == 2 ? 1 : 2;
    };
    std::vector<int2> blk;
    BatchPlan& P = c->bplan;
    P.n_groups = 0;
    for (int g = 0; g < 3; ++g) {
        const int first = (int)blk.size();
        size_t gs = 0;
        for (int q = 0; q < ns; ++q) {
            if (cls(sys_smem[q]) != g) continue;
            gs = std::max(gs, sys_smem[q]);
            for (int w = 0; w < c->sub[q]->W; ++w) blk.push_back(make_int2(q, w));
        }
        if ((int)blk.size() == first) continue;
        P.gfirst[P.n_groups] = first;
        P.gsmem[P.n_groups] = gs;
        P.n_groups++;
        P.gfirst[P.n_groups] = (int)blk.size();
    }
    // fused step: the same groups, systems in decreasing order of work (strings x electrons), so the
    // persistent blocks finish the large ones first and the small ones fill the tail
    std::vector<int2> items;
    for (int g = 0; g < P.n_groups; ++g) {
        std::vector<int> qs;
        for (int b = P.gfirst[g]; b < P.gfirst[g + 1]; ++b)
            if (qs.empty() || qs.back() != blk[b].x) qs.push_back(blk[b].x);
        size_t sm = 0;
        for (int q : qs) {
            const msd_ctx* sc = c->sub[q];
            const size_t chi = (size_t)NCH * sc->nb * sc->tb;
            for (int sp = 0; sp < 2; ++sp)
                sm = std::max(sm, std::max(sys_smem[q], std::max(chi, accept_smem_bytes(sc->sp[sp].n))));
        }
        auto work = [&](int q) {
            const msd_ctx* sc = c->sub[q];
            return (double)(sc->sp[0].g.n_exc + sc->sp[1].g.n_exc) * (sc->sp[0].n + sc->sp[1].n);
        };
        std::stable_sort(qs.begin(), qs.end(), [&](int a, int b) { return work(a) > work(b); });
        for (int q : qs)
            for (int w = 0; w < c->sub[q]->W; ++w) items.push_back(make_int2(q, w));
        P.step_smem[g] = sm;
    }
    BatchSys* d_sys = nullptr;
    int2* d_blk = nullptr;
    int4* d_tiles = nullptr;
    int* d_wsys = nullptr;
    TRY(upload(c, &d_sys, sys.data(), sys.size()));
    TRY(upload(c, &d_blk, blk.data(), blk.size()));
    TRY(upload(c, &d_tiles, tiles.data(), tiles.size()));
    if (!tc_tiles.empty()) {
        int4* d_tc = nullptr;
        TRY(upload(c, &d_tc, tc_tiles.data(), tc_tiles.size()));
        c->bplan.tc_tiles = d_tc;
        c->bplan.n_tc_tiles = (int)tc_tiles.size();
        c->bplan.tc_smem = tc_smem;
    }
    TRY(upload(c, &d_wsys, wsys.data(), wsys.size()));
    {
        int2* d_items = nullptr;
        TRY(upload(c, &d_items, items.data(), items.size()));
        c->bplan.items = d_items;
        std::vector<int> zeros(2 * BatchPlan::kMaxGroups, 0);
        int* d_cnt = nullptr;
        TRY(upload(c, &d_cnt, zeros.data(), zeros.size()));
        c->bplan.counters = d_cnt;
    }
    TRY(dalloc(c, &c->b_rnew, (size_t)c->W * 3));
    c->bplan.sys = d_sys;
    c->bplan.n_sys = ns;
    c->bplan.blk = d_blk;
    c->bplan.n_blk = (int)blk.size();
    c->bplan.tiles = d_tiles;
    c->bplan.n_tiles = (int)tiles.size();
    c->bplan.wsys = d_wsys;
    c->bplan.ratio_smem = rsm;
    c->bplan.accept_smem = asm_;
    return MSD_OK;
}

// Per-system bookkeeping of a batched msd_ratio (refresh, CI weights: launched on the internal
// streams between a fork and a join when a system needs them), then one launch each for the
// orbitals at r' and the ratio of every system.
// Per-system bookkeeping before move `elec` of a batch (refresh every K moves of a spin, CI
// weights when the moving spin changed), on the internal streams; marks the proposal as made.
msd_status batch_prepare(msd_ctx* c, int elec, int nch) {
    bool forked = false;
    for (size_t q = 0; q < c->sub.size(); ++q) {
        msd_ctx* sc = c->sub[q];
        State& st = sc->st;
        if (!st.ready) return fail(c, MSD_ERR_STATE, "system %zu: msd_set_positions has not been called", q);
        const int e = elec % sc->n_tot, s = spin_of(sc, e);
        const bool refresh = st.since_refresh[s] >= sc->K;
        if (refresh || !st.C_valid[s]) {
            if (!forked) {
                TRY(batch_fork(c));
                forked = true;
            }
            msd_status r = MSD_OK;
            if (refresh) {
                r = refresh_spin(sc, st, s);
                if (r == MSD_OK) r = ensure_C(sc, st, s);
                if (r == MSD_OK) r = recompute_S(sc, st, s);
                if (r == MSD_OK) r = rescue_update(sc);
            } else {
                r = ensure_C(sc, st, s);
            }
            if (r != MSD_OK) {
                batch_join(c);
                return fail(c, r, "system %zu: %s", q, sc->err.c_str());
            }
        }
        st.since_refresh[s]++;
        sc->prop_elec = e;
        sc->prop_nch = nch;
        sc->prop_valid = true;
    }
    if (forked) TRY(batch_join(c));
    return MSD_OK;
}

msd_status batch_ratio(msd_ctx* c, int elec, const double* rnew_dev, double* ratio_dev, double* grad_dev,
                       double* lap_dev) {
    if ((grad_dev == nullptr) != (lap_dev == nullptr))
        return fail(c, MSD_ERR_ARG, "grad_dev and lap_dev must be both NULL or both set");
    const int nch = grad_dev ? NCH : 1;
    TRY(batch_prepare(c, elec, nch));
    const cudaError_t e = cudaMemcpyAsync(c->b_rnew, rnew_dev, sizeof(double) * 3 * c->W, cudaMemcpyDeviceToDevice,
                                          c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "copy of rnew: %s", cudaGetErrorString(e));
    if (c->mixed && c->bplan.n_tc_tiles > 0)
        launch_orbitals_tc_batched(c->L(), c->bplan, elec, nch, c->b_rnew);
    else
        launch_orbitals_batched(c->L(), c->mixed, c->bplan, elec, nch, c->b_rnew);
    launch_ratio_batched(c->L_sweep(), c->mixed, c->bplan, elec, nch, ratio_dev, grad_dev, lap_dev);
    TRY(check_launch(c, "batched ratio"));
    if (c->mixed) {
        bool any = false;
        for (msd_ctx* sc : c->sub) any = any || rescue_on(sc);
        if (any) {
            TRY(batch_fork(c));
            for (size_t q = 0; q < c->sub.size(); ++q) {
                msd_ctx* sc = c->sub[q];
                if (!rescue_on(sc)) continue;
                const long long w = c->w_off[q];
                const msd_status r = rescue_ratio(sc, elec % sc->n_tot, rnew_dev + 3 * w, ratio_dev + w,
                                                  grad_dev ? grad_dev + 3 * w : nullptr, lap_dev ? lap_dev + w : nullptr);
                if (r != MSD_OK) {
                    batch_join(c);
                    return fail(c, r, "system %zu: %s", q, sc->err.c_str());
                }
            }
            TRY(batch_join(c));
        }
        launch_check_finite_batched(c->L(), c->bplan, c->W, ratio_dev);
    }
    return check_launch(c, "batched ratio");
}

msd_status batch_accept(msd_ctx* c, int elec, const uint8_t* accept_dev) {
    int nch = 0;
    for (size_t q = 0; q < c->sub.size(); ++q) {
        msd_ctx* sc = c->sub[q];
        const int e = elec % sc->n_tot;
        if (!sc->prop_valid || sc->prop_elec != e)
            return fail(c, MSD_ERR_STATE, "system %zu: msd_accept(%d) without a matching msd_ratio proposal", q, elec);
        nch = sc->prop_nch;
    }
    for (msd_ctx* sc : c->sub) {
        const int s = spin_of(sc, elec % sc->n_tot);
        sc->st.C_valid[1 - s] = false;
        sc->prop_valid = false;
    }
    launch_accept_batched(c->L(), c->mixed, c->bplan, elec, nch, accept_dev, c->b_rnew);
    TRY(check_launch(c, "batched accept"));
    bool any = false;
    for (msd_ctx* sc : c->sub) any = any || rescue_on(sc);
    if (any) {
        TRY(batch_fork(c));
        for (size_t q = 0; q < c->sub.size(); ++q) {
            msd_ctx* sc = c->sub[q];
            if (!rescue_on(sc)) continue;
            const msd_status r = rescue_accept(sc, elec % sc->n_tot, accept_dev + c->w_off[q]);
            if (r != MSD_OK) {
                batch_join(c);
                return fail(c, r, "system %zu: %s", q, sc->err.c_str());
            }
        }
        TRY(batch_join(c));
    }
    return MSD_OK;
}

// Candidate grids of the fused step per group: a persistent grid at the occupancy limit, half of
// it, and one block per item (the counter then hands each block one item).
void step_candidates(msd_ctx* c) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int g = 0; g < c->bplan.n_groups; ++g) {
        const int n = c->bplan.gfirst[g + 1] - c->bplan.gfirst[g];
        const int occ = std::max(1, step_blocks_per_sm(c->mixed, c->bplan.step_smem[g]));
        std::vector<int> cand = {std::min(n, occ * sms), std::min(n, std::max(1, occ * sms / 2)), n};
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        c->tune.candidates[g] = cand;
        c->tune.chosen[g] = cand.front();
    }
}

// One Metropolis step of every system: bookkeeping, then one persistent launch per group (the first
// calls time each candidate grid with events and keep the fastest per group), then the
// finiteness check of the FP32 path.
msd_status batch_step(msd_ctx* c, int elec, const double* eta_dev, double tau, const double* u_dev, double* ratio_dev,
                      double* grad_dev, double* lap_dev, uint8_t* accept_dev) {
    TRY(batch_prepare(c, elec, NCH));
    auto& T = c->tune;
    if (T.candidates[0].empty()) step_candidates(c);
    const bool tuning = !T.done;
    const int k = T.calls;
    if (tuning && !T.ev[0])
        for (int i = 0; i < 2 * BatchPlan::kMaxGroups; ++i) cudaEventCreate(&T.ev[i]);
    for (int g = 0; g < c->bplan.n_groups; ++g) {
        int grid = T.chosen[g];
        if (tuning) grid = T.candidates[g][std::min<size_t>(k, T.candidates[g].size() - 1)];
        if (tuning) cudaEventRecord(T.ev[2 * g], c->stream);
        launch_step_batched(c->L(), c->mixed, c->bplan, g, grid, elec, eta_dev, tau, u_dev, ratio_dev, grad_dev,
                            lap_dev, accept_dev, c->b_rnew);
        if (tuning) cudaEventRecord(T.ev[2 * g + 1], c->stream);
    }
    TRY(check_launch(c, "batched step"));
    if (tuning) {
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "step tuning: %s", cudaGetErrorString(e));
        size_t longest = 0;
        for (int g = 0; g < c->bplan.n_groups; ++g) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, T.ev[2 * g], T.ev[2 * g + 1]);
            if ((size_t)k < T.candidates[g].size()) T.ms[g].push_back(ms);
            longest = std::max(longest, T.candidates[g].size());
        }
        if ((size_t)++T.calls >= longest) {
            for (int g = 0; g < c->bplan.n_groups; ++g) {
                size_t best = 0;
                for (size_t i = 1; i < T.ms[g].size(); ++i)
                    if (T.ms[g][i] < T.ms[g][best]) best = i;
                T.chosen[g] = T.candidates[g][best];
            }
            T.done = true;
        }
    }
    if (c->mixed) launch_check_finite_batched(c->L(), c->bplan, c->W, ratio_dev);
    for (msd_ctx* sc : c->sub) {
        const int s = spin_of(sc, elec % sc->n_tot);
        sc->st.C_valid[1 - s] = false;
        sc->prop_valid = false;
    }
    return check_launch(c, "batched step");
}

msd_status batch_init(const msd_problem* p, int n_systems, msd_ctx** out) {
    for (int s = 0; s < n_systems; ++s) {
        const msd_status st = validate(p + s);
        if (st != MSD_OK) return fail(nullptr, st, "system %d: %s", s, g_init_error.c_str());
    }
    msd_ctx* c = new msd_ctx();
    c->stream = static_cast<cudaStream_t>(p[0].cuda_stream);
    c->mixed = p[0].prec == MSD_MIXED;
    auto bail = [&](msd_status st) {
        const std::string msg = c->err.empty() ? g_init_error : c->err;
        msd_destroy(c);
        g_init_error = msg;
        return st;
    };
    const int ns = std::min(n_systems, kBatchStreams);
    c->bstreams.assign(ns, nullptr);
    c->bevents.assign(ns + 1, nullptr);
    for (int i = 0; i < ns; ++i)
        if (cudaStreamCreateWithFlags(&c->bstreams[i], cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(c, MSD_ERR_CUDA, "stream creation failed"));
    for (int i = 0; i <= ns; ++i)
        if (cudaEventCreateWithFlags(&c->bevents[i], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(c, MSD_ERR_CUDA, "event creation failed"));
    long long w = 0, r = 0, d = 0, b = 0;
    for (int s = 0; s < n_systems; ++s) {
        msd_problem q = p[s];
        q.cuda_stream = c->bstreams[s % ns];
        msd_ctx* sc = nullptr;
        const msd_status st = msd_init(&q, 1, &sc);
        if (st != MSD_OK) return bail(fail(c, st, "system %d: %s", s, g_init_error.c_str()));
        c->sub.push_back(sc);
        c->w_off.push_back(w);
        c->r_off.push_back(r);
        c->det_off.push_back(d);
        c->b_off.push_back(b);
        w += q.n_walkers;
        r += 3LL * q.n_walkers * (q.n_elec[0] + q.n_elec[1]);
        d += q.n_det;
        b += (long long)q.n_basis * (q.n_orb[0] + q.n_orb[1]);
    }
    c->W = (int)w;
    if (dalloc(c, &c->b_status_scratch, 1) != MSD_OK) return bail(MSD_ERR_OOM);
    if (dalloc(c, &c->step_rnew, (size_t)c->W * 3) != MSD_OK) return bail(MSD_ERR_OOM);
    if (build_batch_plan(c) != MSD_OK) return bail(MSD_ERR_CUDA);
    *out = c;
    return MSD_OK;
}

}  // namespace

extern "C" {

msd_status msd_init(const msd_problem* p, int32_t n_systems, msd_ctx** out) {
    g_init_error.clear();
    if (!out) return fail(nullptr, MSD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_systems < 1) return fail(nullptr, MSD_ERR_ARG, "n_systems = %d must be >= 1", n_systems);
    if (!p) return fail(nullptr, MSD_ERR_ARG, "problem is NULL");
    if (n_systems > 1) return batch_init(p, n_systems, out);
    TRY(validate(p));
    msd_ctx* c = new msd_ctx();
    c->W = p->n_walkers;
    c->n_tot = p->n_elec[0] + p->n_elec[1];
    c->nb = p->n_basis;
    c->K = p->refresh_K;
    c->mixed = p->prec == MSD_MIXED;
    c->canon = p->prec == MSD_CANONICAL;
    c->tb = c->mixed ? 4 : 8;
    c->stream = static_cast<cudaStream_t>(p->cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, MSD_ERR_CUDA, "no CUDA device");
    }
    auto bail = [&](msd_status s) {
        g_init_error = c->err;
        msd_destroy(c);
        return s;
    };
    msd_status st;
    if ((st = plan_problem(c->sp, p)) != MSD_OK) {
        c->err = g_init_error;
        return bail(st);
    }
    c->nuc_xyz.assign(p->nuc_xyz, p->nuc_xyz + 3 * (size_t)p->n_nuc);
    // basis
    std::vector<double4> bas(c->nb);
    for (int mu = 0; mu < c->nb; ++mu) {
        const double* A = p->nuc_xyz + 3 * p->bas_center[mu];
        bas[mu] = make_double4(A[0], A[1], A[2], p->bas_alpha[mu]);
    }
    if ((st = upload(c, &c->bas, bas.data(), bas.size())) != MSD_OK) return bail(st);
    if (c->mixed) {
        std::vector<double> cen(3 * (size_t)c->nb);
        for (int mu = 0; mu < c->nb; ++mu)
            for (int i = 0; i < 3; ++i) cen[3 * mu + i] = p->nuc_xyz[3 * p->bas_center[mu] + i];
        std::vector<float4> bf(2 * (size_t)c->nb);
        tc_basis_pairs(c->nb, cen.data(), p->bas_alpha, reinterpret_cast<float*>(bf.data()));
        if ((st = upload(c, &c->basf, bf.data(), bf.size())) != MSD_OK) return bail(st);
    }
    if ((st = upload(c, &c->blm, p->bas_lm, (size_t)c->nb)) != MSD_OK) return bail(st);
    for (int s = 0; s < 2; ++s) {
        SpinConst& S = c->sp[s];
        const size_t cnt = (size_t)c->nb * S.N;
        if (c->mixed) {
            std::vector<float> b32(p->B[s], p->B[s] + cnt);
            float* d = nullptr;
            if ((st = upload(c, &d, b32.data(), cnt)) != MSD_OK) return bail(st);
            S.B = d;
            S.tc = tc_plan(c->nb, S.N);
            if ((st = upload_split_B(c, S, p->B[s])) != MSD_OK) return bail(st);
        } else {
            double* d = nullptr;
            if ((st = upload(c, &d, p->B[s], cnt)) != MSD_OK) return bail(st);
            S.B = d;
        }
        if ((st = upload_spin(c, S)) != MSD_OK) return bail(st);
    }
    const int nmax = std::max(c->sp[0].n, c->sp[1].n);
    const int Nmax = std::max(c->sp[0].N, c->sp[1].N);
    const int mmax = std::max(std::max(c->sp[0].m, c->sp[1].m), 1);
    const size_t W = c->W;
    if ((st = valloc(c, &c->Phi, W * nmax * Nmax * c->tb)) != MSD_OK) return bail(st);
    if ((st = valloc(c, &c->phi_new, W * NCH * Nmax * c->tb)) != MSD_OK) return bail(st);
    if ((st = valloc(c, &c->phi_tmp, W * NCH * Nmax * c->tb)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->rho, W)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->num, W * NCH)) != MSD_OK) return bail(st);
    if ((st = valloc(c, &c->y0, W * mmax * c->tb)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->rnew, W * 3)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->step_rnew, W * 3)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->dummy, W)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->d_io, W * 8)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->d_acc, W)) != MSD_OK) return bail(st);
    if ((st = dalloc(c, &c->d_status, 1)) != MSD_OK) return bail(st);
    if (cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) return bail(fail(c, MSD_ERR_CUDA, "memset"));
    if ((st = alloc_state(c, c->st)) != MSD_OK) return bail(st);
    if ((st = rescue_alloc(c, p)) != MSD_OK) return bail(st);
    if (c->canon) {
        for (int s = 0; s < 2; ++s) {
            const SpinConst& S = c->sp[s];
            std::vector<uint8_t> used(S.g.n_exc);
            for (int j = 0; j < S.g.n_exc; ++j) used[j] = S.user_of[j] >= 0;
            if ((st = upload(c, &c->cn_used[s], used.data(), used.size())) != MSD_OK) return bail(st);
            if ((st = dalloc(c, &c->cn_D[s], (size_t)W * S.g.n_exc * S.n * S.n)) != MSD_OK) return bail(st);
            if ((st = dalloc(c, &c->cn_t[s], (size_t)W * S.g.n_exc)) != MSD_OK) return bail(st);
            if ((st = dalloc(c, &c->cn_ru[s], (size_t)W * S.g.n_exc)) != MSD_OK) return bail(st);
            if ((st = dalloc(c, &c->cn_Phi[s], (size_t)W * S.n * S.N)) != MSD_OK) return bail(st);
        }
    }
    {
        c->n_det = p->n_det;
        std::vector<int> iu(p->n_det), id(p->n_det);
        for (int64_t I = 0; I < p->n_det; ++I) {
            iu[I] = c->sp[0].internal_of[p->det_up[I]];
            id[I] = c->sp[1].internal_of[p->det_dn[I]];
        }
        if ((st = upload(c, &c->term_iu, iu.data(), iu.size())) != MSD_OK) return bail(st);
        if ((st = upload(c, &c->term_id, id.data(), id.size())) != MSD_OK) return bail(st);
    }
    *out = c;
    return MSD_OK;
}

msd_status msd_describe(const msd_problem* p, int64_t* out) {
    g_init_error.clear();
    if (!out) return fail(nullptr, MSD_ERR_ARG, "out is NULL");
    TRY(validate(p));
    SpinConst sp[2];
    TRY(plan_problem(sp, p));
    for (int s = 0; s < 2; ++s) {
        int64_t* o = out + 16 * s;
        o[0] = sp[s].g.n_exc;
        o[1] = sp[s].g.dense1;
        o[2] = sp[s].g.kmax;
        o[3] = sp[s].n_heavy;
        o[4] = (int64_t)sp[s].h_rec.size();
        for (int k = 0; k <= MAXK + 1; ++k) o[5 + k] = sp[s].g.goff[k];
        o[15] = (int64_t)sp[s].h_toff.back();
    }
    return MSD_OK;
}

msd_status msd_describe_records(const msd_problem* p, int32_t spin, uint8_t* out, int64_t cap, int64_t* out_off,
                                int64_t* bytes) {
    g_init_error.clear();
    if (!bytes || !out_off || spin < 0 || spin > 1 || cap < 0) return fail(nullptr, MSD_ERR_ARG, "invalid argument");
    TRY(validate(p));
    SpinConst sp[2];
    TRY(plan_problem(sp, p));
    const SpinConst& S = sp[spin];
    for (int k = 0; k <= MAXK; ++k) out_off[k] = S.g.roff[k];
    out_off[MAXK + 1] = (int64_t)S.h_rec.size();
    *bytes = (int64_t)S.h_rec.size();
    if (out) std::memcpy(out, S.h_rec.data(), (size_t)std::min<int64_t>(cap, *bytes));
    return MSD_OK;
}

msd_status msd_set_positions(msd_ctx* c, const double* R_dev) {
    if (is_batch(c) && R_dev)
        return batch_each(c, [&](int s, msd_ctx* sc) { return msd_set_positions(sc, R_dev + c->r_off[s]); });
    if (!c || !R_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    c->prop_valid = false;
    TRY(rescue_reset(c));
    TRY(set_positions(c, c->st, R_dev));
    return rescue_update(c);
}

msd_status msd_ratio(msd_ctx* c, int32_t elec, const double* rnew_dev, double* ratio_dev, double* grad_dev,
                     double* lap_dev) {
    if (is_batch(c) && rnew_dev && ratio_dev && elec >= 0) return batch_ratio(c, elec, rnew_dev, ratio_dev, grad_dev, lap_dev);
    if (!c || !rnew_dev || !ratio_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (elec < 0 || elec >= c->n_tot) return fail(c, MSD_ERR_ARG, "electron %d out of range", elec);
    if ((grad_dev == nullptr) != (lap_dev == nullptr))
        return fail(c, MSD_ERR_ARG, "grad_dev and lap_dev must be both NULL or both set");
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    if (c->canon) {
        State& st = c->st;
        const int s = spin_of(c, elec);
        const SpinConst& S = c->sp[s];
        if (st.since_refresh[s] >= c->K) {
            TRY(canon_refresh(c, st, s));
            TRY(canon_C(c, st, s, true));
        } else {
            TRY(canon_C(c, st, s, false));
        }
        st.since_refresh[s]++;
        const int nch = grad_dev ? NCH : 1;
        cudaError_t e = cudaMemcpyAsync(c->rnew, rnew_dev, sizeof(double) * c->W * 3, cudaMemcpyDeviceToDevice,
                                        c->stream);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "copy of rnew: %s", cudaGetErrorString(e));
        launch_orbitals(c->L(), false, nch, c->W, 1, c->rnew, 3, 0, c->bas, c->blm, c->nb, S.B, S.N, c->phi_new);
        launch_canon_ratio(c->L_sweep(), c->W, S.n, S.N, S.m, elec - S.off, nch, S.g, c->cn_used[s],
                           static_cast<const double*>(c->phi_new), c->cn_D[s], c->cn_t[s],
                           static_cast<const double*>(st.C[s]), st.S, c->cn_ru[s], ratio_dev, grad_dev, lap_dev,
                           c->num, c->rho);
        TRY(check_launch(c, "canonical ratio"));
        c->prop_elec = elec;
        c->prop_nch = nch;
        c->prop_valid = true;
        return MSD_OK;
    }
    State& st = c->st;
    const int s = spin_of(c, elec);
    const SpinConst& S = c->sp[s];
    if (st.since_refresh[s] >= c->K) {
        TRY(refresh_spin(c, st, s));
        TRY(ensure_C(c, st, s));
        TRY(recompute_S(c, st, s));
        TRY(rescue_update(c));
    } else {
        TRY(ensure_C(c, st, s));
    }
    st.since_refresh[s]++;
    const int nch = grad_dev ? NCH : 1;
    cudaError_t e = cudaMemcpyAsync(c->rnew, rnew_dev, sizeof(double) * c->W * 3, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "copy of rnew: %s", cudaGetErrorString(e));
    orbitals(c, S, nch, c->W, 1, c->rnew, 3, 0, c->phi_new);
    RatioArgs a{};
    a.W = c->W; a.n = S.n; a.N = S.N; a.m = S.m; a.row = elec - S.off; a.nch = nch;
    a.phi = c->phi_new; a.Ainv = st.Ainv[s]; a.T = st.T[s]; a.C = st.C[s]; a.S = st.S; a.g = S.g;
    a.ratio = ratio_dev; a.rs = 1; a.grad = grad_dev; a.gs = 3; a.lap = lap_dev; a.ls = 1;
    a.rho = c->rho; a.num = c->num; a.y0 = c->y0;
    if (S.m == 0) a.g.kmax = 0;
    {
        // while walkers are held in FP64, their FP32 values are overwritten and checked afterwards
        Launch lr = c->L_sweep();
        if (rescue_on(c)) {
            lr.status = c->rs.d_status_scratch;
            TRY(rescue_ratio_begin(c, elec, rnew_dev, grad_dev != nullptr));
        }
        launch_ratio(lr, c->mixed, a);
    }
    TRY(check_launch(c, "ratio"));
    if (rescue_on(c)) TRY(rescue_ratio_end(c, ratio_dev, grad_dev, lap_dev));
    c->prop_elec = elec;
    c->prop_nch = nch;
    c->prop_valid = true;
    return MSD_OK;
}

msd_status msd_accept(msd_ctx* c, int32_t elec, const uint8_t* accept_dev) {
    if (is_batch(c) && accept_dev && elec >= 0) return batch_accept(c, elec, accept_dev);
    if (!c || !accept_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (!c->prop_valid || c->prop_elec != elec)
        return fail(c, MSD_ERR_STATE, "msd_accept(%d) without a matching msd_ratio proposal", elec);
    if (c->canon) {
        State& st = c->st;
        const int s = spin_of(c, elec);
        const SpinConst& S = c->sp[s];
        launch_canon_accept(c->L(), c->W, S.n, S.N, S.m, elec - S.off, elec, c->n_tot, S.g, c->cn_used[s], accept_dev,
                            static_cast<const double*>(c->phi_new), c->prop_nch, c->cn_Phi[s], c->cn_D[s], c->cn_t[s],
                            c->cn_ru[s], c->rnew, st.R, c->rho, c->num, st.logdet[s], st.sgn[s], st.S);
        st.C_valid[1 - s] = false;
        c->prop_valid = false;
        return check_launch(c, "canonical accept");
    }
    State& st = c->st;
    const int s = spin_of(c, elec);
    const SpinConst& S = c->sp[s];
    AcceptArgs a{};
    a.W = c->W; a.n = S.n; a.N = S.N; a.m = S.m; a.row = elec - S.off; a.elec = elec; a.n_tot = c->n_tot;
    a.accept = accept_dev; a.phi = c->phi_new; a.nch = c->prop_nch; a.rho = c->rho; a.num = c->num; a.y0 = c->y0;
    a.rnew = c->rnew; a.Ainv = st.Ainv[s]; a.T = st.T[s]; a.R = st.R; a.logdet = st.logdet[s]; a.sgn = st.sgn[s];
    a.S = st.S;
    if (rescue_on(c)) {
        a.skip = c->rs.d_slot_of;
        TRY(rescue_accept_begin(c, elec, accept_dev));
    }
    launch_accept(c->L(), c->mixed, a);
    st.C_valid[1 - s] = false;
    c->prop_valid = false;
    if (rescue_on(c)) TRY(side_join(c));
    return check_launch(c, "accept");
}

static msd_status grad_lap_main(msd_ctx* c, int32_t elec, double* grad_dev, double* lap_dev);

msd_status msd_grad_lap(msd_ctx* c, int32_t elec, double* grad_dev, double* lap_dev) {
    TRY(grad_lap_main(c, elec, grad_dev, lap_dev));
    if (c && !is_batch(c) && rescue_on(c)) {
        // held walkers: from the FP64 context
        Rescue& r = c->rs;
        TRY(side_fork(c));
        const bool all = elec < 0;
        double* g = all ? r.ga_grad : r.grad;
        double* l = all ? r.ga_lap : r.lap;
        const msd_status st = msd_grad_lap(r.fb, elec, g, l);
        if (st != MSD_OK) return rescue_fail(c, st);
        TRY(side_join(c));
        const int k = all ? c->n_tot : 1;
        launch_scatter_rows(c->L(), r.active, r.d_walker_of, 3 * k, g, grad_dev);
        launch_scatter_rows(c->L(), r.active, r.d_walker_of, k, l, lap_dev);
        return check_launch(c, "rescue grad/lap");
    }
    return MSD_OK;
}

static msd_status grad_lap_main(msd_ctx* c, int32_t elec, double* grad_dev, double* lap_dev) {
    if (c && c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    if (is_batch(c) && grad_dev && lap_dev && elec >= -1)
        return batch_each(c, [&](int s, msd_ctx* sc) {
            // one electron: [W_s][3] per system; all electrons: [W_s][n_tot_s][3] per system
            const long long go = elec >= 0 ? 3 * c->w_off[s] : c->r_off[s];
            const long long lo = elec >= 0 ? c->w_off[s] : c->r_off[s] / 3;
            return msd_grad_lap(sc, elec >= 0 ? sub_elec(c, s, elec) : -1, grad_dev + go, lap_dev + lo);
        });
    if (!c || !grad_dev || !lap_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (elec < -1 || elec >= c->n_tot) return fail(c, MSD_ERR_ARG, "electron %d out of range", elec);
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    if (elec >= 0) return grad_lap_one(c, c->st, elec, grad_dev, 3, lap_dev, 1);
    // every electron at once: the cofactor scatter Tbar of each spin gives the G of a move of
    // any electron i as (A_0^{-T} Tbar)[i], so one sweep per spin replaces n sweeps
    {
        State& st = c->st;
        const size_t W = c->W;
        const int nmax = std::max(c->sp[0].n, c->sp[1].n);
        const int Nmax = std::max(c->sp[0].N, c->sp[1].N);
        const int mmax = std::max(1, std::max(c->sp[0].m, c->sp[1].m));
        if (!c->bw_M) TRY(dalloc(c, &c->bw_M, W * nmax * Nmax));
        if (!c->ga_G) TRY(valloc(c, &c->ga_G, W * nmax * mmax * c->tb));
        if (!c->ga_phid) TRY(valloc(c, &c->ga_phid, W * nmax * NCH * Nmax * c->tb));
        for (int s = 0; s < 2; ++s) {
            const SpinConst& S = c->sp[s];
            if (tbar_smem_bytes(c->mixed, S.n, S.m) > 220 * 1024) {
                // table and its adjoint exceed shared memory: one sweep per electron instead
                for (int e = S.off; e < S.off + S.n; ++e)
                    TRY(grad_lap_one(c, st, e, grad_dev + 3 * e, 3LL * c->n_tot, lap_dev + e, c->n_tot));
                continue;
            }
            TRY(ensure_C(c, st, s));
            launch_tbar(c->L(), c->mixed, c->W, S.n, S.m, S.N, S.g, st.T[s], st.C[s], st.S, c->bw_M);
            orbitals(c, S, NCH, c->W * S.n, S.n, st.R, (long long)c->n_tot * 3, S.off, c->ga_phid);
            launch_all_gradlap(c->L(), c->mixed, c->W, S.n, S.m, S.N, c->n_tot, S.off, st.Ainv[s], st.T[s], c->bw_M,
                               c->ga_phid, c->ga_G, grad_dev, lap_dev);
            TRY(check_launch(c, "all-electron gradient"));
        }
    }
    return MSD_OK;
}

msd_status msd_eval_batch(msd_ctx* c, const double* R_dev, double* logabs_dev, double* sign_dev, double* grad_dev,
                          double* lap_dev) {
    if (c && c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    if (is_batch(c) && R_dev && logabs_dev && sign_dev)
        return batch_each(c, [&](int s, msd_ctx* sc) {
            const long long w = c->w_off[s], r = c->r_off[s];
            return msd_eval_batch(sc, R_dev + r, logabs_dev + w, sign_dev + w, grad_dev ? grad_dev + r : nullptr,
                                  lap_dev ? lap_dev + r / 3 : nullptr);
        });
    if (!c || !R_dev || !logabs_dev || !sign_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if ((grad_dev == nullptr) != (lap_dev == nullptr))
        return fail(c, MSD_ERR_ARG, "grad_dev and lap_dev must be both NULL or both set");
    TRY(alloc_state(c, c->scratch));
    State& st = c->scratch;
    TRY(set_positions(c, st, R_dev));
    launch_state(c->L(), c->W, st.logdet[0], st.sgn[0], st.logdet[1], st.sgn[1], st.S, logabs_dev, sign_dev);
    if (grad_dev)
        for (int e = 0; e < c->n_tot; ++e)
            TRY(grad_lap_one(c, st, e, grad_dev + 3 * e, 3LL * c->n_tot, lap_dev + e, c->n_tot));
    return check_launch(c, "eval_batch");
}

msd_status msd_get_state(msd_ctx* c, double* R_dev, double* logabs_dev, double* sign_dev) {
    if (is_batch(c))
        return batch_each(c, [&](int s, msd_ctx* sc) {
            const long long w = c->w_off[s];
            return msd_get_state(sc, R_dev ? R_dev + c->r_off[s] : nullptr, logabs_dev ? logabs_dev + w : nullptr,
                                 sign_dev ? sign_dev + w : nullptr);
        });
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    State& st = c->st;
    if (R_dev) {
        cudaError_t e = cudaMemcpyAsync(R_dev, st.R, sizeof(double) * c->W * c->n_tot * 3, cudaMemcpyDeviceToDevice,
                                        c->stream);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "copy of positions: %s", cudaGetErrorString(e));
    }
    if (logabs_dev || sign_dev)
        launch_state(c->L(), c->W, st.logdet[0], st.sgn[0], st.logdet[1], st.sgn[1], st.S, logabs_dev, sign_dev);
    if (rescue_on(c) && (logabs_dev || sign_dev)) {
        Rescue& r = c->rs;
        TRY(side_fork(c));
        const msd_status rs_st = msd_get_state(r.fb, nullptr, r.logabs, r.sign);
        if (rs_st != MSD_OK) return rescue_fail(c, rs_st);
        TRY(side_join(c));
        if (logabs_dev) launch_scatter_rows(c->L(), r.active, r.d_walker_of, 1, r.logabs, logabs_dev);
        if (sign_dev) launch_scatter_rows(c->L(), r.active, r.d_walker_of, 1, r.sign, sign_dev);
    }
    return check_launch(c, "get_state");
}

msd_status msd_propose(msd_ctx* c, int32_t elec, const double* eta_dev, double tau, double* rnew_dev) {
    if (is_batch(c) && eta_dev && rnew_dev && elec >= 0) {
        launch_propose_batched(c->L(), c->bplan, c->W, elec, eta_dev, tau, rnew_dev);
        return check_launch(c, "batched proposal");
    }
    if (!c || !eta_dev || !rnew_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (elec < 0 || elec >= c->n_tot) return fail(c, MSD_ERR_ARG, "electron %d out of range", elec);
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    launch_propose(c->L(), c->W, c->n_tot, elec, c->st.R, eta_dev, tau, rnew_dev);
    return check_launch(c, "propose");
}

msd_status msd_metropolis(msd_ctx* c, const double* u_dev, const double* ratio_dev, uint8_t* accept_dev) {
    if (is_batch(c) && u_dev && ratio_dev && accept_dev) {
        launch_metropolis(c->L(), c->W, u_dev, ratio_dev, accept_dev);  // elementwise over all walkers
        return check_launch(c, "metropolis");
    }
    if (!c || !u_dev || !ratio_dev || !accept_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    launch_metropolis(c->L(), c->W, u_dev, ratio_dev, accept_dev);
    return check_launch(c, "metropolis");
}

msd_status msd_step(msd_ctx* c, int32_t elec, const double* eta_dev, double tau, const double* u_dev,
                    double* ratio_dev, double* grad_dev, double* lap_dev, uint8_t* accept_dev) {
    if (!c || !eta_dev || !u_dev || !ratio_dev || !grad_dev || !lap_dev || !accept_dev)
        return fail(c, MSD_ERR_ARG, "NULL argument");
    if (elec < 0) return fail(c, MSD_ERR_ARG, "electron %d out of range", elec);
    if (c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    if (is_batch(c)) {
        bool held = false;
        for (const msd_ctx* sc : c->sub) held = held || rescue_on(sc);
        if (!held) return batch_step(c, elec, eta_dev, tau, u_dev, ratio_dev, grad_dev, lap_dev, accept_dev);
        // walkers held in FP64: the separate calls, which serve them
        TRY(msd_propose(c, elec, eta_dev, tau, c->step_rnew));
        TRY(msd_ratio(c, elec, c->step_rnew, ratio_dev, grad_dev, lap_dev));
        TRY(msd_metropolis(c, u_dev, ratio_dev, accept_dev));
        return msd_accept(c, elec, accept_dev);
    }
    if (elec >= c->n_tot) return fail(c, MSD_ERR_ARG, "electron %d out of range", elec);
    TRY(msd_propose(c, elec, eta_dev, tau, c->step_rnew));
    TRY(msd_ratio(c, elec, c->step_rnew, ratio_dev, grad_dev, lap_dev));
    TRY(msd_metropolis(c, u_dev, ratio_dev, accept_dev));
    return msd_accept(c, elec, accept_dev);
}

msd_status msd_ratio_host(msd_ctx* c, int32_t elec, const double* rnew_host, double* ratio_host, double* grad_host,
                          double* lap_host) {
    if (is_batch(c) && rnew_host && ratio_host && elec >= 0) {
        // host twins run system after system (each call is synchronous)
        for (size_t q = 0; q < c->sub.size(); ++q) {
            const long long w = c->w_off[q];
            const msd_status st = msd_ratio_host(c->sub[q], sub_elec(c, (int)q, elec), rnew_host + 3 * w, ratio_host + w,
                                                 grad_host ? grad_host + 3 * w : nullptr, lap_host ? lap_host + w : nullptr);
            if (st != MSD_OK) return fail(c, st, "system %zu: %s", q, c->sub[q]->err.c_str());
        }
        return MSD_OK;
    }
    if (!c || !rnew_host || !ratio_host) return fail(c, MSD_ERR_ARG, "NULL argument");
    if ((grad_host == nullptr) != (lap_host == nullptr))
        return fail(c, MSD_ERR_ARG, "grad_host and lap_host must be both NULL or both set");
    const size_t W = c->W;
    double* d_rnew = c->d_io;          // [W][3]
    double* d_ratio = c->d_io + 3 * W; // [W]
    double* d_grad = c->d_io + 4 * W;  // [W][3]
    double* d_lap = c->d_io + 7 * W;   // [W]
    cudaError_t e = cudaMemcpyAsync(d_rnew, rnew_host, sizeof(double) * 3 * W, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    TRY(msd_ratio(c, elec, d_rnew, d_ratio, grad_host ? d_grad : nullptr, grad_host ? d_lap : nullptr));
    e = cudaMemcpyAsync(ratio_host, d_ratio, sizeof(double) * W, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && grad_host) {
        e = cudaMemcpyAsync(grad_host, d_grad, sizeof(double) * 3 * W, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lap_host, d_lap, sizeof(double) * W, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "download: %s", cudaGetErrorString(e));
    return MSD_OK;
}

msd_status msd_accept_host(msd_ctx* c, int32_t elec, const uint8_t* accept_host) {
    if (is_batch(c) && accept_host && elec >= 0) {
        for (size_t q = 0; q < c->sub.size(); ++q) {
            const msd_status st = msd_accept_host(c->sub[q], sub_elec(c, (int)q, elec), accept_host + c->w_off[q]);
            if (st != MSD_OK) return fail(c, st, "system %zu: %s", q, c->sub[q]->err.c_str());
        }
        return MSD_OK;
    }
    if (!c || !accept_host) return fail(c, MSD_ERR_ARG, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(c->d_acc, accept_host, c->W, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    TRY(msd_accept(c, elec, c->d_acc));
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "sync: %s", cudaGetErrorString(e));
    return MSD_OK;
}

msd_status msd_set_stream(msd_ctx* c, void* stream) {
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    c->stream = static_cast<cudaStream_t>(stream);
    return MSD_OK;
}

msd_status msd_sync(msd_ctx* c) {
    if (is_batch(c)) {
        for (size_t q = 0; q < c->sub.size(); ++q) {
            const msd_status st = msd_sync(c->sub[q]);
            if (st != MSD_OK) return fail(c, st, "system %zu: %s", q, c->sub[q]->err.c_str());
        }
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
        return MSD_OK;
    }
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    if (c->rs.fb) {
        const msd_status fs = msd_sync(c->rs.fb);
        if (fs != MSD_OK) return rescue_fail(c, fs);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    int status = 0;
    e = cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "status read: %s", cudaGetErrorString(e));
    if (status) {
        cudaMemset(c->d_status, 0, sizeof(int));
        if (status & ST_TIMEOUT)
            return fail(c, MSD_ERR_TIMEOUT, "a bounded wait of a tensor-core kernel gave up (result not written)");
        if (status & ST_SINGULAR) return fail(c, MSD_ERR_SINGULAR, "a reference determinant or ratio was zero");
        return fail(c, MSD_ERR_SINGULAR, "a ratio was not finite");
    }
    return MSD_OK;
}

const char* msd_last_error(const msd_ctx* c) {
    if (!c) return g_init_error.c_str();
    return c->err.c_str();
}

msd_status msd_exc_histogram(const msd_ctx* c, int32_t spin, int64_t* out) {
    if (is_batch(c)) return MSD_ERR_ARG;  // per system: query a single-system context
    if (!c || !out || spin < 0 || spin > 1) return MSD_ERR_ARG;
    out[0] = c->sp[spin].g.n_exc;
    for (int k = 0; k <= MAXK; ++k) out[1 + k] = c->sp[spin].hist[k];
    return MSD_OK;
}

msd_status msd_copy_state(msd_ctx* c, int32_t item, int32_t spin, void* dst, int64_t* bytes) {
    if (is_batch(c)) return fail(c, MSD_ERR_ARG, "msd_copy_state takes a single-system context");
    if (c && c->canon && (item == 1 || item == 2 || item == 7 || item == 10))
        return fail(c, MSD_ERR_ARG, "the canonical method keeps no table state (items Ainv, T, t, y0)");
    if (!c || spin < 0 || spin > 1 || item < 0 || item > 11) return fail(c, MSD_ERR_ARG, "invalid argument");
    if (item >= 8) {
        if (c->prop_elec < 0) return fail(c, MSD_ERR_STATE, "no msd_ratio proposal yet");
        spin = c->prop_elec < c->sp[0].n ? 0 : 1;
    }
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    const State& st = c->st;
    const SpinConst& S = c->sp[spin];
    const size_t W = c->W;
    const void* src = nullptr;
    size_t nb = 0;
    switch (item) {
        case 0: src = st.R; nb = W * c->n_tot * 3 * 8; break;
        case 1: src = st.Ainv[spin]; nb = W * S.n * S.n * 8; break;
        case 2: src = st.T[spin]; nb = W * S.n * S.m * c->tb; break;
        case 3: src = st.logdet[spin]; nb = W * 8; break;
        case 4: src = st.sgn[spin]; nb = W * 8; break;
        case 5: src = st.S; nb = W * 8; break;
        case 6: src = st.C[spin]; nb = W * S.g.n_exc * c->tb; break;
        case 7: src = st.t[spin]; nb = W * S.g.n_exc * c->tb; break;
        case 8: src = c->rho; nb = W * 8; break;
        case 9: src = c->num; nb = W * NCH * 8; break;
        case 10: src = c->y0; nb = W * S.m * c->tb; break;
        case 11: src = c->phi_new; nb = W * c->prop_nch * S.N * c->tb; break;
    }
    if (bytes) *bytes = (int64_t)nb;
    if (dst && nb) {
        cudaError_t e = cudaMemcpyAsync(dst, src, nb, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    }
    return MSD_OK;
}

msd_status msd_timing_start(msd_ctx* c) {
    if (is_batch(c))
        for (msd_ctx* sc : c->sub) TRY(msd_timing_start(sc));  // their own bookkeeping launches; then ours
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    c->timing = true;
    c->launches = 0;
    c->n_refresh = 0;
    c->n_ci = 0;
    c->ev_used = 0;
    return MSD_OK;
}

msd_status msd_timing_counts(const msd_ctx* c, int64_t* out) {
    if (!c || !out) return MSD_ERR_ARG;
    out[0] = c->n_refresh;
    out[1] = c->n_ci;
    for (const msd_ctx* sc : c->sub) {
        out[0] += sc->n_refresh;
        out[1] += sc->n_ci;
    }
    return MSD_OK;
}

msd_status msd_timing_stop(msd_ctx* c, double* sweep_ms, int64_t* sweep_launches, int64_t* all_launches) {
    if (is_batch(c) && c->timing) {
        // the single-launch stages (this context's events) plus the systems' own launches
        double own = 0.0;
        int64_t o1 = 0, o2 = 0;
        c->sub.swap(c->sub_parked);
        const msd_status st0 = msd_timing_stop(c, &own, &o1, &o2);
        c->sub.swap(c->sub_parked);
        TRY(st0);
        double ms = own;
        int64_t n1 = o1, n2 = o2;
        for (msd_ctx* sc : c->sub) {
            double a = 0.0;
            int64_t b = 0, d = 0;
            TRY(msd_timing_stop(sc, &a, &b, &d));
            ms += a;
            n1 += b;
            n2 += d;
        }
        if (sweep_ms) *sweep_ms = ms;
        if (sweep_launches) *sweep_launches = n1;
        if (all_launches) *all_launches = n2;
        return MSD_OK;
    }
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "event time: %s", cudaGetErrorString(e));
        tot += ms;
    }
    if (sweep_ms) *sweep_ms = tot;
    if (sweep_launches) *sweep_launches = (int64_t)(c->ev_used / 2);
    if (all_launches) *all_launches = c->launches;
    c->timing = false;
    c->ev_used = 0;
    return MSD_OK;
}

msd_status msd_set_hamiltonian(msd_ctx* c, const double* Z_host, const msd_jastrow* jas) {
    if (is_batch(c)) return fail(c, MSD_ERR_ARG, "msd_set_hamiltonian takes a single-system context");
    if (!c || !Z_host) return fail(c, MSD_ERR_ARG, "NULL argument");
    const int n_nuc = (int)(c->nuc_xyz.size() / 3);
    const double b_ee = jas ? jas->b_ee : 0.0, b_en = jas ? jas->b_en : 0.0;
    if (!std::isfinite(b_ee) || !std::isfinite(b_en) || b_ee < 0.0 || b_en < 0.0)
        return fail(c, MSD_ERR_ARG, "Jastrow parameters must be finite and >= 0 (0 = term absent)");
    std::vector<double4> nuc(n_nuc);
    for (int I = 0; I < n_nuc; ++I) {
        const double Z = Z_host[I];
        if (!std::isfinite(Z) || Z < 0.0) return fail(c, MSD_ERR_ARG, "charge of nucleus %d must be finite and >= 0", I);
        const double* A = c->nuc_xyz.data() + 3 * I;
        nuc[I] = make_double4(A[0], A[1], A[2], Z);
    }
    // nuclear repulsion sum_{I<J} Z_I Z_J / R_IJ (a constant of the clamped nuclei)
    double vnn = 0.0;
    for (int I = 0; I < n_nuc; ++I)
        for (int J = I + 1; J < n_nuc; ++J) {
            const double dx = nuc[I].x - nuc[J].x, dy = nuc[I].y - nuc[J].y, dz = nuc[I].z - nuc[J].z;
            const double zz = nuc[I].w * nuc[J].w;
            if (zz == 0.0) continue;
            const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (r == 0.0) return fail(c, MSD_ERR_ARG, "charged nuclei %d and %d coincide", I, J);
            vnn += zz / r;
        }
    // the kernels of earlier calls may still read the charges: wait before overwriting them
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, MSD_ERR_CUDA, "stream synchronisation failed");
    if (!c->ham_nuc) TRY(dalloc(c, &c->ham_nuc, (size_t)n_nuc));
    if (cudaMemcpy(c->ham_nuc, nuc.data(), sizeof(double4) * n_nuc, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(c, MSD_ERR_CUDA, "upload of the nuclear charges failed");
    c->ham_b_ee = b_ee;
    c->ham_b_en = b_en;
    c->ham_vnn = vnn;
    c->ham_set = true;
    return MSD_OK;
}

}  // extern "C"

namespace {
msd::HamArgs ham_args(const msd_ctx* c) {
    msd::HamArgs a;
    a.W = c->W;
    a.n_tot = c->n_tot;
    a.n_up = c->sp[0].n;
    a.n_nuc = (int)(c->nuc_xyz.size() / 3);
    a.R = c->st.R;
    a.nuc = c->ham_nuc;
    a.b_ee = c->ham_b_ee;
    a.b_en = c->ham_b_en;
    a.vnn = c->ham_vnn;
    return a;
}
}  // namespace

extern "C" {

msd_status msd_jastrow_ratio(msd_ctx* c, int32_t elec, const double* rnew_dev, double* ratio_dev) {
    if (is_batch(c)) return fail(c, MSD_ERR_ARG, "msd_jastrow_ratio takes a single-system context");
    if (!c || !rnew_dev || !ratio_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (elec < 0 || elec >= c->n_tot) return fail(c, MSD_ERR_ARG, "electron %d out of range", elec);
    if (!c->ham_set) return fail(c, MSD_ERR_STATE, "msd_set_hamiltonian has not been called");
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    launch_jastrow_ratio(c->L(), ham_args(c), elec, rnew_dev, ratio_dev);
    return check_launch(c, "Jastrow ratio");
}

msd_status msd_local_energy(msd_ctx* c, double* eloc_dev, double* parts_dev) {
    if (c && c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    if (is_batch(c)) return fail(c, MSD_ERR_ARG, "msd_local_energy takes a single-system context");
    if (!c || !eloc_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (!c->ham_set) return fail(c, MSD_ERR_STATE, "msd_set_hamiltonian has not been called");
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    const size_t W = c->W;
    if (!c->le_grad) TRY(dalloc(c, &c->le_grad, W * c->n_tot * 3));
    if (!c->le_lap) TRY(dalloc(c, &c->le_lap, W * c->n_tot));
    TRY(msd_grad_lap(c, -1, c->le_grad, c->le_lap));
    launch_local_energy(c->L(), ham_args(c), c->le_grad, c->le_lap, eloc_dev, parts_dev);
    return check_launch(c, "local energy");
}

void msd_destroy(msd_ctx* c) {
    if (c && !c->sub.empty()) {
        for (msd_ctx* sc : c->sub) msd_destroy(sc);
        c->sub.clear();
    }
    if (c) {
        for (cudaStream_t st : c->bstreams)
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t ev : c->bevents)
            if (ev) cudaEventDestroy(ev);
        c->bstreams.clear();
        c->bevents.clear();
    }
    if (!c) return;
    if (c->rs.fb) {
        msd_destroy(c->rs.fb);
        c->rs.fb = nullptr;
    }
    if (c->rs.side) {
        cudaStreamSynchronize(c->rs.side);
        cudaStreamDestroy(c->rs.side);
        cudaEventDestroy(c->rs.ev_fork);
        cudaEventDestroy(c->rs.ev_join);
    }
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->tune.ev)
        if (e) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

msd_status msd_ratio_noalloc(msd_ctx* c, int32_t elec, const double* rnew_dev, double* ratio_dev, double* grad_dev,
                             double* lap_dev) {
    if (c && c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    if (is_batch(c))  // its scratch is one array per device: systems on concurrent streams would share it
        return fail(c, MSD_ERR_ARG, "msd_ratio_noalloc takes a single-system context");
    if (!c || !rnew_dev || !ratio_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (elec < 0 || elec >= c->n_tot) return fail(c, MSD_ERR_ARG, "electron %d out of range", elec);
    if ((grad_dev == nullptr) != (lap_dev == nullptr))
        return fail(c, MSD_ERR_ARG, "grad_dev and lap_dev must be both NULL or both set");
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    State& st = c->st;
    const int s = spin_of(c, elec);
    const SpinConst& S = c->sp[s];
    const int nch = grad_dev ? NCH : 1;
    const size_t need = (size_t)c->W * nch * S.N * c->tb;
    if (need > kNoAllocScratchBytes)
        return fail(c, MSD_ERR_ARG,
                    "msd_ratio_noalloc needs %zu bytes of scratch (walkers x channels x orbitals x %d bytes), "
                    "above its fixed limit of %zu bytes; use msd_ratio",
                    need, c->tb, kNoAllocScratchBytes);
    // the scratch array is looked up for the current device: it must be the context's own
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev != c->device)
        return fail(c, MSD_ERR_ARG, "msd_ratio_noalloc: current device %d is not the context's device %d", dev,
                    c->device);
    void* phi = nullptr;
    e = noalloc_scratch(&phi);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "scratch address: %s", cudaGetErrorString(e));
    TRY(ensure_C(c, st, s));
    orbitals(c, S, nch, c->W, 1, rnew_dev, 3, 0, phi);
    RatioArgs a{};
    a.W = c->W; a.n = S.n; a.N = S.N; a.m = S.m; a.row = elec - S.off; a.nch = nch;
    a.phi = phi; a.Ainv = st.Ainv[s]; a.T = st.T[s]; a.C = st.C[s]; a.S = st.S; a.g = S.g;
    a.ratio = ratio_dev; a.rs = 1; a.grad = grad_dev; a.gs = 3; a.lap = lap_dev; a.ls = 1;
    a.rho = nullptr; a.num = nullptr; a.y0 = nullptr;
    if (S.m == 0) a.g.kmax = 0;
    launch_ratio(c->L(), c->mixed, a);
    return check_launch(c, "ratio (no allocation)");
}

msd_status msd_set_rescue(msd_ctx* c, int32_t slots, double kappa_hold, double kappa_release) {
    if (is_batch(c)) {
        for (size_t q = 0; q < c->sub.size(); ++q) {
            const msd_status st = msd_set_rescue(c->sub[q], slots, kappa_hold, kappa_release);
            if (st != MSD_OK) return fail(c, st, "system %zu: %s", q, c->sub[q]->err.c_str());
        }
        return MSD_OK;
    }
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    if (!c->mixed) return fail(c, MSD_ERR_ARG, "only the mixed-precision path holds walkers in FP64");
    if (slots < 0 || slots > c->rs.slots_max())
        return fail(c, MSD_ERR_ARG, "slots = %d outside [0, %d]", slots, c->rs.slots_max());
    if (!(kappa_hold > 1.0) || !(kappa_release > 1.0) || !(kappa_release <= kappa_hold))
        return fail(c, MSD_ERR_ARG, "need 1 < kappa_release <= kappa_hold");
    Rescue& r = c->rs;
    TRY(rescue_reset(c));
    if (r.fb && slots != r.slots) {  // its walker count is the slot count
        msd_destroy(r.fb);
        r.fb = nullptr;
    }
    r.slots = slots;
    r.k_demote = kappa_hold;
    r.k_promote = kappa_release;
    if (c->st.ready) return rescue_update(c);  // from the condition estimates of the last refreshes
    return MSD_OK;
}

msd_status msd_rescue_stats(const msd_ctx* c, int64_t* out) {
    if (!c || !out) return MSD_ERR_ARG;
    for (int i = 0; i < 5; ++i) out[i] = 0;
    auto add = [&](const msd_ctx* x) {
        out[0] += x->rs.active;
        out[1] += x->rs.demotions;
        out[2] += x->rs.promotions;
        out[3] += x->rs.overflow;
        out[4] += x->rs.slots;
    };
    if (!c->sub.empty())
        for (const msd_ctx* sc : c->sub) add(sc);
    else
        add(c);
    return MSD_OK;
}

msd_status msd_selftest_wait(msd_ctx* c, int64_t wait_ns) {
    if (is_batch(c)) return fail(c, MSD_ERR_ARG, "msd_selftest_wait takes a single-system context");
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    if (wait_ns < 1000 || wait_ns > 1000000000) return fail(c, MSD_ERR_ARG, "wait_ns = %lld outside [1e3, 1e9]",
                                                            (long long)wait_ns);
    launch_wait_selftest(c->L(), (unsigned long long)wait_ns);
    return check_launch(c, "wait self-test");
}

msd_status msd_orbitals(msd_ctx* c, int32_t spin, int32_t nch, int32_t n_points, const double* pos_dev,
                        void* out_dev) {
    if (is_batch(c)) return fail(c, MSD_ERR_ARG, "msd_orbitals takes a single-system context");
    if (!c || !pos_dev || !out_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (spin < 0 || spin > 1) return fail(c, MSD_ERR_ARG, "spin %d is not 0 or 1", spin);
    if (nch != 1 && nch != NCH) return fail(c, MSD_ERR_ARG, "nch = %d must be 1 or 5", nch);
    if (n_points < 0) return fail(c, MSD_ERR_ARG, "n_points = %d < 0", n_points);
    if (c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    orbitals(c, c->sp[spin], nch, n_points, 1, pos_dev, 3, 0, out_dev);
    return check_launch(c, "orbitals");
}

msd_status msd_backward(msd_ctx* c, const double* gbar_dev, double* dci_dev, double* dB_dev) {
    if (c && c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    if (is_batch(c) && gbar_dev && dci_dev && dB_dev)
        return batch_each(c, [&](int q, msd_ctx* sc) {
            return msd_backward(sc, gbar_dev + c->w_off[q], dci_dev + c->det_off[q], dB_dev + c->b_off[q]);
        });
    if (!c || !gbar_dev || !dci_dev || !dB_dev) return fail(c, MSD_ERR_ARG, "NULL argument");
    if (!c->st.ready) return fail(c, MSD_ERR_STATE, "msd_set_positions has not been called");
    for (int s = 0; s < 2; ++s) {
        const SpinConst& S = c->sp[s];
        if (tbar_smem_bytes(c->mixed, S.n, S.m) > 220 * 1024)
            return fail(c, MSD_ERR_ARG, "spin %d: table and its adjoint (%d x %d) do not fit in shared memory", s, S.n,
                        S.m);
    }
    State& st = c->st;
    const size_t W = c->W;
    const int nmax = std::max(c->sp[0].n, c->sp[1].n);
    const int Nmax = std::max(c->sp[0].N, c->sp[1].N);
    if (!c->bw_M) TRY(dalloc(c, &c->bw_M, W * nmax * Nmax));
    if (!c->bw_chi) TRY(dalloc(c, &c->bw_chi, W * nmax * c->nb));
    // every quantity from scratch at the current positions (as msd_set_positions does)
    c->prop_valid = false;
    TRY(refresh_spin(c, st, 0));
    TRY(refresh_spin(c, st, 1));
    st.C_valid[0] = st.C_valid[1] = false;
    TRY(ensure_C(c, st, 0));     // t_dn, C_up
    TRY(recompute_S(c, st, 0));  // t_up, S
    TRY(ensure_C(c, st, 1));     // C_dn
    cudaError_t e = cudaMemsetAsync(dci_dev, 0, sizeof(double) * c->n_det, c->stream);
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    launch_dci(c->L(), c->mixed, c->W, c->n_det, c->term_iu, c->term_id, gbar_dev, st.S, st.t[0], c->sp[0].g.n_exc,
               st.t[1], c->sp[1].g.n_exc, dci_dev);
    double* dB = dB_dev;
    for (int s = 0; s < 2; ++s) {
        const SpinConst& S = c->sp[s];
        launch_phibar(c->L(), c->mixed, c->W, S.n, S.m, S.N, S.g, st.T[s], st.C[s], st.S, st.Ainv[s], gbar_dev,
                      c->bw_M);
        launch_chi(c->L(), c->W * S.n, S.n, st.R, (long long)c->n_tot * 3, S.off, c->bas, c->blm, c->nb, c->bw_chi);
        e = cudaMemsetAsync(dB, 0, sizeof(double) * c->nb * S.N, c->stream);
        if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
        launch_dB(c->L(), c->W * S.n, c->nb, S.N, c->bw_chi, c->bw_M, dB);
        dB += (size_t)c->nb * S.N;
    }
    return check_launch(c, "backward");
}

msd_status msd_set_params(msd_ctx* c, const double* ci_host, const double* B_up_host, const double* B_dn_host) {
    if (c && c->canon) return fail(c, MSD_ERR_ARG, "not available for the canonical method");
    if (is_batch(c)) {
        for (size_t q = 0; q < c->sub.size(); ++q) {
            const msd_ctx* sc = c->sub[q];
            const double* b = B_up_host ? B_up_host + c->b_off[q] : nullptr;
            const double* bd = b ? b + (size_t)sc->nb * sc->sp[0].N : nullptr;
            const msd_status st =
                msd_set_params(c->sub[q], ci_host ? ci_host + c->det_off[q] : nullptr, b, bd);
            if (st != MSD_OK) return fail(c, st, "system %zu: %s", q, c->sub[q]->err.c_str());
        }
        return MSD_OK;
    }
    if (!c) return fail(c, MSD_ERR_ARG, "NULL context");
    if ((B_up_host == nullptr) != (B_dn_host == nullptr))
        return fail(c, MSD_ERR_ARG, "B_up_host and B_dn_host must be both NULL or both set");
    if (ci_host)
        for (long long I = 0; I < c->n_det; ++I)
            if (!std::isfinite(ci_host[I])) return fail(c, MSD_ERR_ARG, "ci[%lld] not finite", I);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
        SpinConst& S = c->sp[s];
        if (ci_host) {
            std::vector<double> cc(c->n_det);
            for (long long I = 0; I < c->n_det; ++I) cc[S.h_tpos[I]] = ci_host[I];
            e = cudaMemcpy(S.t_c, cc.data(), sizeof(double) * cc.size(), cudaMemcpyHostToDevice);
        }
        if (B_up_host && e == cudaSuccess) {
            const double* Bh = s ? B_dn_host : B_up_host;
            const size_t cnt = (size_t)c->nb * S.N;
            if (c->mixed) {
                std::vector<float> b32(Bh, Bh + cnt);
                e = cudaMemcpy(S.B, b32.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice);
                if (e == cudaSuccess && S.Bsplit) {
                    const msd_status r = upload_split_B(c, S, Bh);
                    if (r != MSD_OK) return r;
                }
            } else {
                e = cudaMemcpy(S.B, Bh, sizeof(double) * cnt, cudaMemcpyHostToDevice);
            }
        }
    }
    if (e != cudaSuccess) return fail(c, MSD_ERR_CUDA, "parameter upload: %s", cudaGetErrorString(e));
    if (c->rs.enabled) {
        // the FP64 context, and the copy it is built from, take the same parameters
        if (ci_host) std::copy(ci_host, ci_host + c->n_det, c->rs.prob.ci.begin());
        if (B_up_host) {
            std::copy(B_up_host, B_up_host + c->rs.prob.B0.size(), c->rs.prob.B0.begin());
            std::copy(B_dn_host, B_dn_host + c->rs.prob.B1.size(), c->rs.prob.B1.begin());
        }
        if (c->rs.fb) {
            const msd_status fs = msd_set_params(c->rs.fb, ci_host, B_up_host, B_dn_host);
            if (fs != MSD_OK) return rescue_fail(c, fs);
        }
    }
    c->prop_valid = false;
    c->scratch.C_valid[0] = c->scratch.C_valid[1] = false;
    if (!c->st.ready) return MSD_OK;
    TRY(rebuild(c, c->st));
    return rescue_update(c);
}

}  // extern "C"
