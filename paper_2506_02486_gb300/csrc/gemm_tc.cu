// gemm_tc.cu -- the block products of Cannon's ring steps (section 5, matrix
// multiplication): C_q = A_q * B_q^T for a set of problems q, BF16 operands,
// FP32 accumulation, on the 5th-generation tensor cores.
//
// One persistent CTA per SM, six warps, one CTA per output tile (no
// clusters):
//   warp 0      TMA producer: (128 MH) x 64 A and 256 x 64 B tiles
//               (K-major, 128-byte swizzle) into a ring of shared-memory
//               stages;
//   warp 1      allocates 512 tensor-memory columns and issues tcgen05.mma
//               (M 128, N 256, K 16), MH products per K slice, all reading
//               the same B stage;
//   warps 2-5   epilogue: tensor memory -> registers -> C.
// MH = 1: 128 x 256 tiles, 4 stages of 48 KB, two accumulators, so the
// epilogue of one tile runs while the next tile is multiplied.  MH = 2:
// 256 x 256 tiles, 3 stages of 64 KB, one pair of accumulators (the two
// M halves); a K step then brings 64 KB from L2 for twice the products,
// 128 instead of 85 multiply-adds per operand byte.
// Every wait is bounded; a wait that gives up latches ERRB_TIMEOUT, the CTA
// drains what it has in flight (bounded), frees its tensor memory and leaves.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "gw_kernels.h"
#include "tc_ptx.cuh"

namespace gw {
namespace {

constexpr int BH = 128, BN = 256, BK = 64;     // M half, N, K depth of a stage
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 2 * BN;         // 512: the whole tensor memory

template <int MH_>
struct Shape {
    static constexpr int MH = MH_;
    static constexpr int BMT = BH * MH;                  // tile rows
    static constexpr int STAGES = MH == 1 ? 4 : 3;
    static constexpr int NACC = MH == 1 ? 2 : 1;         // accumulator sets
    static constexpr int A_BYTES = BMT * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    // barriers: full[S], empty[S], tfull[NACC], tempty[NACC], drain; then
    // the TMEM base address and an abort flag
    static constexpr int OFF_BAR = STAGES * STAGE_BYTES;
    static constexpr int NBAR = 2 * STAGES + 2 * NACC + 1;
    static constexpr int OFF_TMEM = OFF_BAR + 8 * NBAR;
    static constexpr int SMEM_BYTES = OFF_TMEM + 16 + 1024;   // + ring alignment
    static_assert(SMEM_BYTES <= 232448, "shared memory");
    static_assert(NACC * MH * BN == (int)TMEM_COLS, "tensor memory");
};

struct TileCoord {
    int q, tm, tn;
};

// Tile t of the launch: problems one after another; inside a problem,
// groups of `group` tile rows swept column by column, so the CTAs running
// at the same time share A rows and B columns in L2, and the next wave
// reuses the group's A rows.
__device__ __forceinline__ TileCoord tile_of(int t, int tmc, int tnc, int group)
{
    const int per = tmc * tnc;
    TileCoord c;
    c.q = t / per;
    const int u = t - c.q * per;
    const int g = u / (group * tnc);
    const int first = g * group;
    const int gs = min(group, tmc - first);
    const int v = u - g * group * tnc;
    c.tm = first + v % gs;
    c.tn = v / gs;
    return c;
}

__device__ __forceinline__ bool bwait(uint64_t *bar, uint32_t parity, volatile int *abortf,
                                      unsigned long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0) {
            if (*abortf) return false;
            if (global_timer() - t0 > limit) return false;
        }
    }
}

// The same bound without the abort shortcut: draining copies and MMAs that
// are already in flight must not be cut short by another warp giving up.
__device__ __forceinline__ bool bwait_drain(uint64_t *bar, uint32_t parity,
                                            unsigned long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0 && global_timer() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void give_up(volatile int *abortf, unsigned *err)
{
    if (!*abortf) atomicOr(err, ERRB_TIMEOUT);
    *abortf = 1;
}

// Tile t of the launch is tile_of(t) (problems one after another, groups
// of `group` tile rows swept column by column); CTA b takes tiles
// b, b + grid, ....  Accumulator set of a CTA's local tile l: l % NACC,
// used for the (l / NACC)-th time.
template <int MH>
__global__ void __launch_bounds__(THREADS, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap map_a,
            const __grid_constant__ CUtensorMap map_b,
            const __grid_constant__ GemmArgs A)
{
    using SH = Shape<MH>;
    constexpr int STAGES = SH::STAGES, NACC = SH::NACC, BMT = SH::BMT,
                  A_BYTES = SH::A_BYTES, STAGE_BYTES = SH::STAGE_BYTES;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment: the swizzle pattern repeats every 8 rows of 128 B
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SH::OFF_BAR);
    uint64_t *full = bars, *empty = bars + STAGES;
    uint64_t *tfull = bars + 2 * STAGES, *tempty = tfull + NACC, *drain = tempty + NACC;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SH::OFF_TMEM);
    volatile int *abortf = reinterpret_cast<volatile int *>(smem + SH::OFF_TMEM + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tmc = (A.m + BMT - 1) / BMT, tnc = (A.n + BN - 1) / BN;
    const int ntiles = A.nprob * tmc * tnc;
    const int nkb = (A.k + BK - 1) / BK;
    const int group = max(1, A.group);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);        // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        *abortf = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const uint64_t pol = policy_evict_normal();
            uint32_t it = 0;
            // (the self-test issues no loads, so that the waits run out)
            for (int t = blockIdx.x; t < ntiles && !A.skip_loads; t += gridDim.x) {
                const TileCoord tc_ = tile_of(t, tmc, tnc, group);
                const int ra = A.a_rank[tc_.q], rb = A.b_rank[tc_.q];
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t s = it % STAGES;
                    if (it >= STAGES &&
                        !bwait(&empty[s], ((it / STAGES) - 1) & 1u, abortf, A.wait_ns)) {
                        give_up(abortf, A.err);
                        goto produced;
                    }
                    unsigned char *st = smem + s * STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_3d(st, &map_a, &full[s], kb * BK, tc_.tm * BMT, ra, pol);
                    tma_load_3d(st + A_BYTES, &map_b, &full[s], kb * BK, tc_.tn * BN, rb, pol);
                }
            }
        produced:
            // leave only after the copies issued into shared memory landed
            for (uint32_t q = it > STAGES ? it - STAGES : 0; q < it; ++q)
                if (!bwait_drain(&full[q % STAGES], (q / STAGES) & 1u, A.wait_ns)) break;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(BH, BN);
            uint32_t it = 0, local = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++local) {
                const uint32_t b = local % NACC, use = local / NACC;
                if (use >= 1 && !bwait(&tempty[b], (use - 1) & 1u, abortf, A.wait_ns)) {
                    give_up(abortf, A.err);
                    break;
                }
                tc::fence_after_sync();
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t s = it % STAGES;
                    if (!bwait(&full[s], (it / STAGES) & 1u, abortf, A.wait_ns)) {
                        give_up(abortf, A.err);
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const unsigned char *st = smem + s * STAGE_BYTES;
                    const uint64_t bd = tc::sdesc_k128(st + A_BYTES);
#pragma unroll
                    for (int h = 0; h < MH; ++h) {
                        // M half h: rows 128 h .. of the A stage (16 KB, a
                        // whole number of 1024-byte swizzle atoms further)
                        const uint64_t ad = tc::sdesc_k128(st + h * (BH * BK * 2));
                        const uint32_t d = tmem + (b * MH + h) * BN;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)   // 32 bytes along K each
                            tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc,
                                         (kb | kk) != 0);
                    }
                    tc::commit(&empty[s]);                 // stage free when done
                }
                if (!ok) break;
                tc::commit(&tfull[b]);                     // accumulators ready
            }
            // no MMA may still be running when the CTA leaves
            tc::commit(drain);
            bwait_drain(drain, 0, A.wait_ns);
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int lg = warp & 3;                  // TMEM lane group of this warp
        const int row_in_half = 32 * lg + lane;
        uint32_t local = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++local) {
            const uint32_t b = local % NACC, use = local / NACC;
            if (!bwait(&tfull[b], use & 1u, abortf, A.wait_ns)) {
                give_up(abortf, A.err);
                break;
            }
            tc::fence_after_sync();
            const TileCoord tc_ = tile_of(t, tmc, tnc, group);
            const int col0 = tc_.tn * BN;
#pragma unroll 1
            for (int h = 0; h < MH; ++h) {
                const int row = tc_.tm * BMT + h * BH + row_in_half;
                float *crow = A.c + A.c_off[tc_.q] + (long long)row * A.ldc + col0;
                const bool vec = ((reinterpret_cast<uintptr_t>(crow) & 15u) == 0);
                const uint32_t tcol = tmem + ((uint32_t)(32 * lg) << 16) + (b * MH + h) * BN;
#pragma unroll 1
                for (int ch = 0; ch < BN / 32; ++ch) {
                    float v[32];
                    tc::ld_32cols(tcol + ch * 32, v);     // whole warp, every row
                    if (row >= A.m) continue;
                    const int c0 = col0 + ch * 32;
                    float *p = crow + ch * 32;
                    if (vec && c0 + 32 <= A.n) {
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            *reinterpret_cast<float4 *>(p + i) =
                                make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (c0 + i < A.n) p[i] = v[i];
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

int gemm_tile_n() { return BN; }

template <int MH>
static cudaError_t set_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<MH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Shape<MH>::SMEM_BYTES);
    done = e == cudaSuccess;
    return e;
}

template <int MH>
static int max_ctas(int num_sms)
{
    if (set_attr<MH>() != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm_bf16<MH>, THREADS,
                                                      Shape<MH>::SMEM_BYTES) != cudaSuccess)
        return 0;
    return per_sm >= 1 ? num_sms : 0;   // one CTA per SM: it holds all TMEM
}

template <int MH>
static cudaError_t launch(const CUtensorMap &ma, const CUtensorMap &mb, const GemmArgs &a,
                          int grid, cudaStream_t s)
{
    cudaError_t e = set_attr<MH>();
    if (e != cudaSuccess) return e;
    k_gemm_bf16<MH><<<grid, THREADS, Shape<MH>::SMEM_BYTES, s>>>(ma, mb, a);
    return cudaGetLastError();
}

int gemm_max_ctas(int tile_m, int num_sms)
{
    switch (tile_m) {
    case 128: return max_ctas<1>(num_sms);
    case 256: return max_ctas<2>(num_sms);
    default: return 0;
    }
}

cudaError_t launch_gemm_bf16(const void *map_a, const void *map_b, const GemmArgs &a,
                             int tile_m, int grid, cudaStream_t s)
{
    CUtensorMap ma, mb;
    memcpy(&ma, map_a, sizeof ma);
    memcpy(&mb, map_b, sizeof mb);
    switch (tile_m) {
    case 128: return launch<1>(ma, mb, a, grid, s);
    case 256: return launch<2>(ma, mb, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gw
