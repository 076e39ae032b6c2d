// msd_tc.cu -- the dense contractions of the FP32 path on the fifth-generation tensor cores of
// sm_103a (tcgen05 MMA with the accumulator in tensor memory): the orbital product and the
// excitation table.
//
// Orbitals.  Algorithm 1 step 2 evaluates the orbitals at a position: phi^a_j(r) = sum_mu chi^a_mu(r) B[mu][j]
// for the value and derivative channels a.  Over P points this is one dense product
//   out[P NC x N] = X[P NC x nb] . B[nb x N],   row p NC + a of X = chi^a(r_p),
// the only dense contraction on the per-move path; the refresh (NC = 1, every electron of a spin)
// and the all-electron gradient (NC = 5, every electron) are the same product with more rows.
//
// Precision: each FP32 operand is split exactly into three TF32 pieces x = x0 + x1 + x2 (11 + 11
// + the remaining bits), and the product keeps the six piece products whose size is at least
// 2^-22 of the whole (x0 y0, x0 y1, x1 y0, x1 y1, x0 y2, x2 y0).  The dropped terms are below
// 2^-32 relative, so with the FP32 accumulator in tensor memory the result carries FP32
// accuracy; B is split from its FP64 value on the host.
//
// Tile: 128 rows (one MMA M: 128 points of one channel, or 25 points x 5 channels) x TN <= 256
// columns per CTA, basis functions in chunks of 8 (one MMA K for kind::tf32) through two
// shared-memory stages.  Per chunk one thread starts a bulk copy (cp.async.bulk, completion counted
// on an mbarrier) of the chunk's pre-split B, the 256 threads evaluate the chunk's basis functions
// at the tile's points (each point once for all its channels) and store the three pieces of X, and
// the same thread issues the six MMAs and commits them to the stage's mbarrier; a stage is refilled
// once the MMAs that read it have completed.  Operands use the K-major layout without swizzle: 8-row x 16-byte core
// matrices, the two K halves of a row group adjacent (leading-dimension offset 128 B), row
// groups 256 B apart (stride offset).  Every wait is bounded in time: on expiry the kernel sets
// ST_TIMEOUT, skips its output, releases its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "msd_basis.cuh"
#include "msd_internal.h"

namespace msd {
namespace {

constexpr int kTcM = 128;           // rows per tile (MMA M), one per thread
constexpr int kTcK = 8;             // basis functions per chunk (MMA K of kind::tf32)
constexpr int kTcParts = 3;         // TF32 pieces per operand
constexpr int kTcThreads = 256;
constexpr int kTcStages = 3;      // operand stages in shared memory
constexpr int kTcABytes = kTcM * kTcK * 4;  // one piece of the X chunk: 4096 B
constexpr unsigned long long kTcWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start address, leading- and stride-dimension byte offsets
// (each >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, N and M.
__host__ __device__ constexpr uint32_t tf32_idesc(int n, int m) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase of the given parity to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kTcWaitNs) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of element (row, k) of a K-major no-swizzle operand chunk of 8 K values:
// row group g = row / 8 at g * 256, K half k / 4 at + 128, row in group at + 16 (row % 8), + 4 (k % 4).
__host__ __device__ constexpr uint32_t kmajor_offset(int row, int k) {
    return (uint32_t)((row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Points per tile: NC = 5 packs 25 points x 5 channels into the 128 MMA rows (3 rows stay zero),
// so the basis functions of a point are evaluated once for all its channels.
template <int NC>
__host__ __device__ constexpr int tc_points_per_tile() {
    return NC == 1 ? kTcM : kTcM / NC;
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// One 128-row x TN-column output tile (tile bx of the points, column tile by) of one product.
template <int NC>
__device__ __forceinline__ void orbitals_tc_tile(int P, int ppw, const double* __restrict__ pos, long long wstride,
                                                 int p_off, const float4* __restrict__ bas,
                                                 const int8_t* __restrict__ blm, int nb,
                                                 const float* __restrict__ Bsplit, int N, int TN,
                                                 float* __restrict__ out, int* __restrict__ status, int bx, int by) {
    constexpr int PPT = tc_points_per_tile<NC>();
    constexpr int QB = (PPT + 7) / 8;           // blocks of 8 points
    constexpr int ITEMS = QB * 2 * 32;          // (8 points x 4 basis functions) per warp item
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2 * kTcStages];  // [s]: MMAs of stage s done; [S + s]: its B landed
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nK = (nb + kTcK - 1) / kTcK;
    const uint32_t b_bytes = (uint32_t)TN * kTcK * 4;  // one piece of the B chunk
    const uint32_t stage_bytes = kTcParts * (kTcABytes + b_bytes);
    const uint32_t ncols = TN <= 32 ? 32u : TN <= 64 ? 64u : TN <= 128 ? 128u : 256u;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t mdone = smem_u32(&mbar[0]), bfull = smem_u32(&mbar[kTcStages]);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2 * kTcStages; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mdone + 8 * i) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // rows of the tile that no point fills (25 x 5 = 125 of 128) stay zero in every stage
    if (PPT * NC < kTcM)
        for (int i = tid; i < kTcStages * kTcParts * (kTcM - PPT * NC) * kTcK; i += kTcThreads) {
            const int k = i % kTcK, rr = PPT * NC + (i / kTcK) % (kTcM - PPT * NC), rest = i / (kTcK * (kTcM - PPT * NC));
            const int piece = rest % kTcParts, st = rest / kTcParts;
            *reinterpret_cast<float*>(smem + st * stage_bytes + piece * kTcABytes + kmajor_offset(rr, k)) = 0.0f;
        }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    const int p0 = bx * PPT;
    const int n0 = by * TN;
    // the tile's points as FP32 (hi, lo) pairs, and the basis centres likewise (bas: centre hi and
    // the exponent, then centre lo): d = (r_hi - A_hi) + (r_lo - A_lo) carries FP32 accuracy relative
    // to |r - A| with no FP64 arithmetic per basis function
    __shared__ float ptile[kTcM][6];
    for (int q = tid; q < PPT; q += kTcThreads) {
        const int pt = p0 + q;
        double x[3] = {0.0, 0.0, 0.0};
        if (pt < P) {
            const int w = pt / ppw;
            const double* rp = pos + (long long)w * wstride + (long long)(p_off + pt - w * ppw) * 3;
            x[0] = rp[0];
            x[1] = rp[1];
            x[2] = rp[2];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float hi = float(x[i]);
            ptile[q][i] = hi;
            ptile[q][3 + i] = float(x[i] - double(hi));
        }
    }
    __syncthreads();
    const float* Bt = Bsplit + (size_t)by * nK * kTcParts * TN * kTcK;
    const uint32_t id = tf32_idesc(TN, kTcM);
    uint32_t mphase = 0u, bphase = 0u;  // bit s: parity of the next phase of stage s
    bool ok = true, ok0 = true;         // ok0: thread 0's own waits (B copies, stage reuse)
    int issued = 0, consumed = 0;       // B copies thread 0 started / saw land
    if (tid == 0)  // B of the first chunks ahead of everything else
        for (; issued < min(nK, kTcStages - 1); ++issued)
            bulk_copy_g2s(sbase + (issued % kTcStages) * stage_bytes + kTcParts * kTcABytes,
                          Bt + (size_t)issued * kTcParts * TN * kTcK, kTcParts * b_bytes,
                          bfull + 8 * (issued % kTcStages));
    for (int kc = 0; kc < nK; ++kc) {
        const int s = kc % kTcStages;
        unsigned char* st = smem + s * stage_bytes;
        bool mine = ok0;
        if (kc >= kTcStages) {
            // the MMAs of chunk kc - kTcStages read this stage: one thread waits, the barrier below
            // orders everyone's writes after its observation
            if (tid == 0) mine = mbar_wait(mdone + 8 * s, (mphase >> s) & 1u) && mine;
            mphase ^= 1u << s;
        }
        ok = __syncthreads_and(mine) != 0;  // the block agrees, so a timeout leaves the loop uniformly
        if (!ok) break;
        // X chunk: basis functions kc 8 .. kc 8 + 7 of the tile's points, all channels, in three TF32
        // pieces.  A warp item covers 8 points x 4 basis functions, so each of its stores fills the 32
        // distinct banks of one 8-row x 16-byte core matrix (5 q mod 8 runs over all residues).
        for (int it = tid; it < ITEMS; it += kTcThreads) {
            const int g = it >> 5, l = it & 31;
            const int q = 8 * (g % QB) + (l & 7), j = 4 * (g / QB) + (l >> 3);
            const int mu = kc * kTcK + j, pt = p0 + q;
            float v[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (q < PPT && pt < P && mu < nb) {
                const float4 ch = bas[2 * mu], cl = bas[2 * mu + 1];
                const float d[3] = {(ptile[q][0] - ch.x) + (ptile[q][3] - cl.x), (ptile[q][1] - ch.y) + (ptile[q][4] - cl.y),
                                    (ptile[q][2] - ch.z) + (ptile[q][5] - cl.z)};
                basis_from_disp<float>(d, ch.w, blm[mu], v);
            }
            if (q < PPT) {
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const float x = v[a];
                    const float h = tf32_rna(x);
                    const float rem = x - h;
                    const float m = tf32_rna(rem);
                    const uint32_t off = kmajor_offset(q * NC + a, j);
                    *reinterpret_cast<float*>(st + 0 * kTcABytes + off) = h;
                    *reinterpret_cast<float*>(st + 1 * kTcABytes + off) = m;
                    *reinterpret_cast<float*>(st + 2 * kTcABytes + off) = tf32_rna(rem - m);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && ok0) {
            ok0 = mbar_wait(bfull + 8 * s, (bphase >> s) & 1u);
            if (ok0) {
                bphase ^= 1u << s;
                ++consumed;
            }
            if (ok0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = sbase + s * stage_bytes;
                const uint32_t sb = sa + kTcParts * kTcABytes;
                // piece pairs (X piece, B piece) whose product is at least 2^-22 of the whole
                const int pa[6] = {0, 0, 1, 1, 0, 2};
                const int pb[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const uint64_t ad = smem_desc(sa + pa[q] * kTcABytes, 128, 256);
                    const uint64_t bd = smem_desc(sb + pb[q] * b_bytes, 128, 256);
                    mma_tf32(tmem, ad, bd, id, (kc > 0 || q > 0) ? 1u : 0u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 mdone + 8 * s)
                             : "memory");
            }
            // B of chunk kc + S - 1 into the stage the MMAs of chunk kc - 1 read, once they are done
            if (ok0 && issued < nK) {
                const int sn = issued % kTcStages;
                if (issued >= kTcStages) {
                    // the stage's previous MMAs (chunk issued - S = kc - 1); all threads later wait on
                    // the same phase at the loop head, so its parity bit is left for them to flip
                    ok0 = mbar_wait(mdone + 8 * sn, (mphase >> sn) & 1u);
                }
                if (ok0) {
                    bulk_copy_g2s(sbase + sn * stage_bytes + kTcParts * kTcABytes,
                                  Bt + (size_t)issued * kTcParts * TN * kTcK, kTcParts * b_bytes, bfull + 8 * sn);
                    ++issued;
                }
            }
        }
    }
    if (ok) ok = __syncthreads_and(ok0) != 0;
    // the last commit covers every MMA issued before it
    if (ok && nK > 0) {
        const int s = (nK - 1) % kTcStages;
        ok = __syncthreads_and(tid == 0 ? mbar_wait(mdone + 8 * s, (mphase >> s) & 1u) : true) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // accumulator rows are TMEM lanes; warp w reads lanes 32 (w % 4) .. + 31 of the 32-column
        // blocks of parity w / 4, stages them in shared memory (the operand stages are free now) and
        // every warp then writes whole 128-byte row segments
        float* stg = reinterpret_cast<float*>(smem);  // [2 blocks][128 rows][33]
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int ncol = min(TN, N - n0);
        const long long row0 = (long long)p0 * NC;
        const long long rows = min((long long)PPT * NC, (long long)P * NC - row0);
        for (int cb0 = 0; cb0 < ncol; cb0 += 64) {
            const int cb = cb0 + 32 * (warp >> 2);
            if (cb < ncol) {
                uint32_t v[32];
                tmem_ld32(tmem + lane_base + (uint32_t)cb, v);
                float* dst = stg + ((warp >> 2) * 128 + 32 * (warp & 3) + lane) * 33;
#pragma unroll
                for (int j = 0; j < 32; ++j) dst[j] = __uint_as_float(v[j]);
            }
            __syncthreads();
            for (int rr = warp; rr < 2 * 128; rr += kTcThreads / 32) {
                const int blk = rr >> 7, row = rr & 127, col = cb0 + 32 * blk + lane;
                if (row < rows && col < ncol) out[(row0 + row) * N + n0 + col] = stg[(blk * 128 + row) * 33 + lane];
            }
            __syncthreads();
        }
    } else {
        if (tid == 0) {
            atomicOr(status, ST_TIMEOUT);
            // before the shared memory goes: the B copies and the MMAs still in flight (bounded)
            for (int c = consumed; c < issued; ++c) {
                const int sc = c % kTcStages;
                mbar_wait(bfull + 8 * sc, (bphase >> sc) & 1u);
                bphase ^= 1u << sc;
            }
        }
        if (tid == 0 && nK > 0) mbar_wait(mdone + 8 * ((nK - 1) % kTcStages), (mphase >> ((nK - 1) % kTcStages)) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

template <int NC>
__global__ void __launch_bounds__(kTcThreads) k_orbitals_tc(int P, int ppw, const double* __restrict__ pos,
                                                           long long wstride, int p_off,
                                                           const float4* __restrict__ bas,
                                                           const int8_t* __restrict__ blm, int nb,
                                                           const float* __restrict__ Bsplit, int N, int TN,
                                                           float* __restrict__ out, int* __restrict__ status) {
    orbitals_tc_tile<NC>(P, ppw, pos, wstride, p_off, bas, blm, nb, Bsplit, N, TN, out, status, blockIdx.x,
                         blockIdx.y);
}

// Batched systems: tile (system, point tile, column tile) of the orbitals at the proposed positions
// of move t (electron t mod n_tot of each system, whose spin selects B).
template <int NC>
__global__ void __launch_bounds__(kTcThreads) k_orbitals_tc_batched(const BatchSys* __restrict__ sys,
                                                                   const int4* __restrict__ tiles, int t,
                                                                   const double* __restrict__ rnew) {
    const int4 tl = tiles[blockIdx.x];
    const BatchSys& B = sys[tl.x];
    const int e = t % B.n_tot;
    const OrbArgs& o = B.orb[e < B.n_up ? 0 : 1];
    if (tl.y * tc_points_per_tile<NC>() >= B.W || tl.z >= o.nT) return;  // uniform over the block
    orbitals_tc_tile<NC>(B.W, 1, rnew + 3LL * B.w_off, 3, 0, o.basf, o.blm, o.nb, o.Bsplit, o.N, o.TN,
                         static_cast<float*>(o.out), B.status, tl.y, tl.z);
}

// A wait that runs out on purpose: an mbarrier that expects one arrival nobody makes, waited on
// with the bounded wait of the tensor-core kernels; on expiry the same status bit is set.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = __syncthreads_and(threadIdx.x == 0 ? mbar_wait(b, 0u, limit_ns) : true) != 0;
    if (!ok && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

// ------------------------------------------------------------------------------------------
// Excitation table T = A_0^{-1} Phi_virt (Algorithm 1 step 3: one matrix product per walker)
// ------------------------------------------------------------------------------------------
// Computed transposed, D[a][c] = T[c][a] = sum_r Phi[r][n + a] Ainv[c][r]: M = virtual orbitals
// (128 per tile), N = occupied orbitals (n rounded up to 16, <= 256), K = electrons r in chunks
// of 32.  Both operands are staged by the threads in three TF32 pieces of their FP32 values
// (A_0^{-1} rounded to FP32, as the FP32 table is stored); the six piece products of size
// >= 2^-22 accumulate in tensor memory, so the product has FP32 accuracy.  The epilogue writes
// rows c of T with consecutive lanes on consecutive a (coalesced).
constexpr int kTbK = 32;                      // electrons per chunk
constexpr int kTbABytes = kTcM * kTbK * 4;    // one piece of the Phi_virt^T chunk: 16 KB

__host__ __device__ constexpr uint32_t kmajor32_offset(int row, int k) {
    return (uint32_t)((row >> 3) * (kTbK * 32) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void split3(float x, float& p0, float& p1, float& p2) {
    p0 = tf32_rna(x);
    const float r = x - p0;
    p1 = tf32_rna(r);
    p2 = tf32_rna(r - p1);
}

__global__ void __launch_bounds__(kTcThreads) k_table_tc(int n, int N, int NP, const double* __restrict__ Ainv,
                                                        const float* __restrict__ Phi, float* __restrict__ T,
                                                        int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int m = N - n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w = blockIdx.y, a0 = blockIdx.x * kTcM;
    const uint32_t b_bytes = (uint32_t)NP * kTbK * 4;
    const uint32_t ncols = NP <= 32 ? 32u : NP <= 64 ? 64u : NP <= 128 ? 128u : 256u;
    const uint32_t sbase = smem_u32(smem), bar = smem_u32(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const double* Aw = Ainv + (long long)w * n * n;
    const float* Pw = Phi + (long long)w * n * N;
    const uint32_t id = tf32_idesc(NP, kTcM);
    const int nK = (n + kTbK - 1) / kTbK;
    uint32_t phase = 0u;
    bool ok = true;
    for (int kc = 0; kc < nK && ok; ++kc) {
        const int r0 = kc * kTbK;
        // A: rows a (virtual orbitals of the tile), K = electrons r: Phi[r][n + a].  A warp covers 8
        // rows x 4 electrons, so each store fills the 32 banks of one core matrix.
        for (int i = tid; i < kTcM * kTbK; i += kTcThreads) {
            const int g = i >> 5, l = i & 31;
            const int row = 8 * (g % (kTcM / 8)) + (l & 7), k = 4 * (g / (kTcM / 8)) + (l >> 3);
            const int a = a0 + row, r = r0 + k;
            const float x = (a < m && r < n) ? Pw[(long long)r * N + n + a] : 0.0f;
            float p0, p1, p2;
            split3(x, p0, p1, p2);
            const uint32_t off = kmajor32_offset(row, k);
            *reinterpret_cast<float*>(smem + off) = p0;
            *reinterpret_cast<float*>(smem + kTbABytes + off) = p1;
            *reinterpret_cast<float*>(smem + 2 * kTbABytes + off) = p2;
        }
        // B: rows c (occupied orbitals), K = electrons r: A_0^{-1}[c][r] rounded to FP32 (the table is
        // stored in FP32) and split there; same warp layout as A
        unsigned char* sbp = smem + 3 * kTbABytes;
        for (int i = tid; i < NP * kTbK; i += kTcThreads) {
            const int g = i >> 5, l = i & 31;
            const int c = 8 * (g % (NP / 8)) + (l & 7), k = 4 * (g / (NP / 8)) + (l >> 3), r = r0 + k;
            const float v = (c < n && r < n) ? float(Aw[(long long)c * n + r]) : 0.0f;
            float p0, p1, p2;
            split3(v, p0, p1, p2);
            const uint32_t off = kmajor32_offset(c, k);
            *reinterpret_cast<float*>(sbp + off) = p0;
            *reinterpret_cast<float*>(sbp + b_bytes + off) = p1;
            *reinterpret_cast<float*>(sbp + 2 * b_bytes + off) = p2;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int pa[6] = {0, 0, 1, 1, 0, 2};
            const int pb[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
            for (int st = 0; st < kTbK / kTcK; ++st)
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const uint64_t ad = smem_desc(sbase + pa[q] * kTbABytes + st * 256, 128, kTbK * 32);
                    const uint64_t bd = smem_desc(sbase + 3 * kTbABytes + pb[q] * b_bytes + st * 256, 128, kTbK * 32);
                    mma_tf32(tmem, ad, bd, id, (kc > 0 || st > 0 || q > 0) ? 1u : 0u);
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        // the next chunk overwrites the operands: wait for these MMAs (one thread, then the block)
        ok = __syncthreads_and(tid == 0 ? mbar_wait(bar, phase) : true) != 0;
        phase ^= 1u;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // lanes are virtual orbitals a; warp w takes column blocks of parity w / 4
        const int a = a0 + 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        float* Tw = T + (long long)w * n * m;
        for (int cb = 32 * (warp >> 2); cb < NP; cb += 64) {
            uint32_t v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)cb, v);
            if (a < m)
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (cb + j < n) Tw[(long long)(cb + j) * m + a] = __uint_as_float(v[j]);
        }
    } else if (tid == 0) {
        atomicOr(status, ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

float host_tf32(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;  // round half away from zero on the dropped 13 bits
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

}  // namespace

void tc_basis_pairs(int nb, const double* centers, const double* alpha, float* out) {
    for (int mu = 0; mu < nb; ++mu) {
        float* hi = out + 8 * mu;
        float* lo = hi + 4;
        for (int i = 0; i < 3; ++i) {
            hi[i] = float(centers[3 * mu + i]);
            lo[i] = float(centers[3 * mu + i] - double(hi[i]));
        }
        hi[3] = float(alpha[mu]);
        lo[3] = 0.0f;
    }
}

TcPlan tc_plan(int nb, int N) {
    TcPlan t;
    const int nT = (N + 255) / 256;
    t.nT = nT;
    t.TN = ((N + nT - 1) / nT + 31) / 32 * 32;
    t.nK = (nb + kTcK - 1) / kTcK;
    t.floats = (size_t)t.nT * t.nK * kTcParts * t.TN * kTcK;
    t.smem = (size_t)kTcStages * kTcParts * (kTcABytes + (size_t)t.TN * kTcK * 4);
    // the epilogue stages two 32-column blocks of 128 rows (33 floats a row) in the same memory
    if (t.smem < (size_t)2 * 128 * 33 * 4) t.smem = (size_t)2 * 128 * 33 * 4;
    // at most two tiles per SM: two accumulators of up to 256 columns fill tensor memory
    if (t.smem < 80 * 1024) t.smem = 80 * 1024;
    return t;
}

void tc_split_B(const TcPlan& t, int nb, int N, const double* B, float* out) {
    std::memset(out, 0, t.floats * sizeof(float));
    for (int tile = 0; tile < t.nT; ++tile)
        for (int kc = 0; kc < t.nK; ++kc)
            for (int j = 0; j < t.TN; ++j) {
                const int col = tile * t.TN + j;
                for (int k = 0; k < kTcK; ++k) {
                    const int mu = kc * kTcK + k;
                    double v = (col < N && mu < nb) ? B[(size_t)mu * N + col] : 0.0;
                    float* base = out + ((size_t)tile * t.nK + kc) * kTcParts * t.TN * kTcK;
                    for (int q = 0; q < kTcParts; ++q) {
                        const float piece = host_tf32(float(v));
                        v -= double(piece);
                        base[(size_t)q * t.TN * kTcK + kmajor_offset(j, k) / 4] = piece;
                    }
                }
            }
}

void launch_orbitals_tc(const Launch& L, int nch, int P, int ppw, const double* pos, long long wstride, int p_off,
                        const float4* bas, const int8_t* blm, int nb, const TcPlan& t, const float* Bsplit, int N,
                        float* out) {
    if (P <= 0 || N <= 0) return;
    const int ppt = nch == 5 ? tc_points_per_tile<5>() : tc_points_per_tile<1>();
    const dim3 grid((unsigned)((P + ppt - 1) / ppt), (unsigned)t.nT);
    L.count();
    if (nch == 5) {
        cudaFuncSetAttribute(k_orbitals_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem);
        k_orbitals_tc<5><<<grid, kTcThreads, t.smem, L.stream>>>(P, ppw, pos, wstride, p_off, bas, blm, nb, Bsplit,
                                                                 N, t.TN, out, L.status);
    } else {
        cudaFuncSetAttribute(k_orbitals_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem);
        k_orbitals_tc<1><<<grid, kTcThreads, t.smem, L.stream>>>(P, ppw, pos, wstride, p_off, bas, blm, nb, Bsplit,
                                                                 N, t.TN, out, L.status);
    }
}

int tc_tile_points(int nch) { return nch == 5 ? tc_points_per_tile<5>() : tc_points_per_tile<1>(); }

void launch_orbitals_tc_batched(const Launch& L, const BatchPlan& P, int t, int nch, const double* rnew) {
    if (P.n_tc_tiles <= 0) return;
    L.count();
    if (nch == 5) {
        cudaFuncSetAttribute(k_orbitals_tc_batched<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.tc_smem);
        k_orbitals_tc_batched<5><<<P.n_tc_tiles, kTcThreads, P.tc_smem, L.stream>>>(P.sys, P.tc_tiles, t, rnew);
    } else {
        cudaFuncSetAttribute(k_orbitals_tc_batched<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.tc_smem);
        k_orbitals_tc_batched<1><<<P.n_tc_tiles, kTcThreads, P.tc_smem, L.stream>>>(P.sys, P.tc_tiles, t, rnew);
    }
}

void launch_wait_selftest(const Launch& L, unsigned long long limit_ns) {
    L.count();
    k_wait_selftest<<<1, 32, 0, L.stream>>>(limit_ns, L.status);
}

bool table_tc_supported(int n) { return n >= 1 && n <= 256; }

void launch_table_tc(const Launch& L, int W, int n, int N, const double* Ainv, const float* Phi, float* T) {
    const int m = N - n;
    if (m <= 0 || W <= 0) return;
    const int NP = (n + 15) / 16 * 16;
    const size_t sm = (size_t)3 * kTbABytes + (size_t)3 * NP * kTbK * 4;
    const dim3 grid((unsigned)((m + kTcM - 1) / kTcM), (unsigned)W);
    L.count();
    cudaFuncSetAttribute(k_table_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_table_tc<<<grid, kTcThreads, sm, L.stream>>>(n, N, NP, Ainv, Phi, T, L.status);
}

}  // namespace msd
