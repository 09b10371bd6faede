// gemm_tc.cu -- the block products of Cannon's ring steps (section 5, matrix
// multiplication): C_q = A_q * B_q^T for a set of problems q, BF16 operands,
// FP32 accumulation, on the 5th-generation tensor cores.
//
// One persistent CTA per SM, six warps:
//   warp 0      TMA producer: 128 x 64 A and 256 x 64 B tiles (K-major,
//               128-byte swizzle) into a 4-stage shared-memory ring;
//   warp 1      allocates 512 tensor-memory columns (two 128 x 256 FP32
//               accumulators) and issues tcgen05.mma (M 128, N 256, K 16);
//   warps 2-5   epilogue: tensor memory -> registers -> C, while the MMA
//               warp fills the other accumulator.
// Every wait is bounded; a wait that gives up latches ERRB_TIMEOUT, the CTA
// drains what it has in flight (bounded), frees its tensor memory and leaves.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "gw_kernels.h"
#include "tc_ptx.cuh"

namespace gw {
namespace {

constexpr int BM = 128, BN = 256;
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 2 * BN;          // two accumulators

// Stage shape for a K depth of BK BF16 per stage: 64 (128-byte rows,
// 128-byte swizzle, 4 stages of 48 KB) or 32 (64-byte rows, 64-byte
// swizzle, 9 stages of 24 KB: the same bytes in flight, refilled in finer
// steps, so the loads run further ahead of the MMAs).
template <int BK_>
struct Shape {
    static constexpr int BK = BK_;
    static constexpr int STAGES = BK == 64 ? 4 : 9;
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    // barriers: full[S], empty[S], tfull[2], tempty[2], drain; then the
    // TMEM base address and an abort flag
    static constexpr int OFF_BAR = STAGES * STAGE_BYTES;
    static constexpr int NBAR = 2 * STAGES + 5;
    static constexpr int OFF_TMEM = OFF_BAR + 8 * NBAR;
    static constexpr int SMEM_BYTES = OFF_TMEM + 16 + 1024;   // + ring alignment
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

// Operand descriptor of a K-major tile of rows of BK BF16 (see tc_ptx.cuh).
template <int BK>
__device__ __forceinline__ uint64_t sdesc(const void *tile)
{
    return BK == 64 ? tc::sdesc_k128(tile) : tc::sdesc_k64(tile);
}

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

// Clusters of CM x CN CTAs on a CM x CN block of tiles (CTA rank
// ci + CM * cj takes tile row tm0 + ci, tile column tn0 + cj).  The CN CTAs
// of a tile row share its A tile and the CM CTAs of a tile column its B
// tile: each CTA loads 1/CN of its A tile and 1/CM of its B tile and
// multicasts them to the CTAs sharing them, so with 2 x 1 a CTA fetches
// 32 KB per K step from L2 and with 2 x 2 24 KB instead of 48 KB.  A stage
// may only be refilled once every CTA that writes into it is done with it:
// each MMA warp's commit arrives on the empty barrier of itself and of the
// CTAs that share its tiles (count CM + CN - 1).
template <int CM, int CN, int BK_>
__global__ void __launch_bounds__(THREADS, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap map_a,
            const __grid_constant__ CUtensorMap map_b,
            const __grid_constant__ GemmArgs A)
{
    using SH = Shape<BK_>;
    constexpr int BK = SH::BK, STAGES = SH::STAGES, A_BYTES = SH::A_BYTES,
                  B_BYTES = SH::B_BYTES, STAGE_BYTES = SH::STAGE_BYTES;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment: the swizzle pattern repeats every 8 rows of 128 B
    // (the same offset in every CTA, as multicast requires)
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SH::OFF_BAR);
    uint64_t *full = bars, *empty = bars + STAGES;
    uint64_t *tfull = bars + 2 * STAGES, *tempty = tfull + 2, *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + SH::OFF_TMEM);
    volatile int *abortf = reinterpret_cast<volatile int *>(smem + SH::OFF_TMEM + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int CL = CM * CN;
    const int crank = CL > 1 ? (int)tc::cluster_ctarank() : 0;
    const int ci = crank % CM, cj = crank / CM;
    const int unit0 = CL > 1 ? (int)tc::cluster_id_x() : (int)blockIdx.x;
    const int nunit_step = CL > 1 ? (int)tc::ncluster_x() : (int)gridDim.x;
    const int tmc = (A.m + BM - 1) / BM, tnc = (A.n + BN - 1) / BN;
    const int tmu = (tmc + CM - 1) / CM;          // unit rows
    const int tnu = (tnc + CN - 1) / CN;          // unit columns
    const int nunits = A.nprob * tmu * tnu;
    const int nkb = (A.k + BK - 1) / BK;
    const int group_u = max(1, A.group / CM);     // unit rows per raster group
    // CTAs sharing this CTA's A tile (same ci) and its B tile (same cj)
    uint16_t row_peers = 0, col_peers = 0;
#pragma unroll
    for (int j = 0; j < CN; ++j) row_peers |= (uint16_t)(1u << (ci + CM * j));
#pragma unroll
    for (int i = 0; i < CM; ++i) col_peers |= (uint16_t)(1u << (i + CM * cj));
    const uint16_t writers = row_peers | col_peers;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CM + CN - 1);   // one commit per writer
        }
        for (int b = 0; b < 2; ++b) {
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
    if (CL > 1) tc::cluster_sync();          // peers' barriers exist
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const uint64_t pol = policy_evict_normal();
            uint32_t it = 0;
            // (the self-test issues no loads, so that the waits run out)
            for (int u = unit0; u < nunits && !A.skip_loads; u += nunit_step) {
                const TileCoord tc_ = tile_of(u, tmu, tnu, group_u);
                const int tm = tc_.tm * CM + ci, tn = tc_.tn * CN + cj;
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
                    if (CN == 1)
                        tma_load_3d(st, &map_a, &full[s], kb * BK, tm * BM, ra, pol);
                    else
                        tc::tma_load_3d_mc(st + cj * (A_BYTES / CN), &map_a, &full[s],
                                           kb * BK, tm * BM + cj * (BM / CN), ra,
                                           row_peers, pol);
                    if (CM == 1)
                        tma_load_3d(st + A_BYTES, &map_b, &full[s], kb * BK, tn * BN, rb, pol);
                    else
                        tc::tma_load_3d_mc(st + A_BYTES + ci * (B_BYTES / CM), &map_b,
                                           &full[s], kb * BK, tn * BN + ci * (BN / CM), rb,
                                           col_peers, pol);
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
            constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
            uint32_t it = 0, local = 0;
            for (int u = unit0; u < nunits; u += nunit_step, ++local) {
                const uint32_t b = local & 1u;
                if (local >= 2 && !bwait(&tempty[b], ((local >> 1) - 1) & 1u, abortf, A.wait_ns)) {
                    give_up(abortf, A.err);
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + b * BN;
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
                    const uint64_t ad = sdesc<BK>(st);
                    const uint64_t bd = sdesc<BK>(st + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)   // 32 bytes along K each
                        tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc,
                                     (kb | kk) != 0);
                    // stage free (in every CTA that wrote into it) when done
                    if (CL == 1) tc::commit(&empty[s]);
                    else tc::commit_mc(&empty[s], writers);
                }
                if (!ok) break;
                tc::commit(&tfull[b]);                     // accumulator ready
            }
            // no MMA may still be running when the CTA leaves
            tc::commit(drain);
            bwait_drain(drain, 0, A.wait_ns);
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int lg = warp & 3;                  // TMEM lane group of this warp
        const int row_in_tile = 32 * lg + lane;
        uint32_t local = 0;
        for (int u = unit0; u < nunits; u += nunit_step, ++local) {
            const uint32_t b = local & 1u;
            if (!bwait(&tfull[b], (local >> 1) & 1u, abortf, A.wait_ns)) {
                give_up(abortf, A.err);
                break;
            }
            tc::fence_after_sync();
            const TileCoord tc_ = tile_of(u, tmu, tnu, group_u);
            const int row = (tc_.tm * CM + ci) * BM + row_in_tile;
            const int col0 = (tc_.tn * CN + cj) * BN;
            float *crow = A.c + A.c_off[tc_.q] + (long long)row * A.ldc + col0;
            const bool vec = ((reinterpret_cast<uintptr_t>(crow) & 15u) == 0);
#pragma unroll 1
            for (int ch = 0; ch < BN / 32; ++ch) {
                float v[32];
                tc::ld_32cols(tmem + ((uint32_t)(32 * lg) << 16) + b * BN + ch * 32, v);
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
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }

    tc::fence_before_sync();
    __syncthreads();
    // a peer may still multicast into this CTA or arrive on its barriers
    // until it has drained its own copies and MMAs
    if (CL > 1) tc::cluster_sync();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

int gemm_tile_m() { return BM; }
int gemm_tile_n() { return BN; }

template <int CM, int CN, int BK>
static cudaError_t set_attr()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<CM, CN, BK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Shape<BK>::SMEM_BYTES);
    done = e == cudaSuccess;
    return e;
}

static cudaLaunchConfig_t config(int cl, int grid, int smem, cudaStream_t s,
                                 cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int CM, int CN, int BK>
static int max_ctas(int num_sms)
{
    constexpr int CL = CM * CN;
    if (set_attr<CM, CN, BK>() != cudaSuccess) return 0;
    if (CL == 1) return num_sms;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = config(CL, CL * (num_sms / CL), Shape<BK>::SMEM_BYTES, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_gemm_bf16<CM, CN, BK>, &cfg) != cudaSuccess)
        return 0;
    return CL * n;
}

template <int CM, int CN, int BK>
static cudaError_t launch(const CUtensorMap &ma, const CUtensorMap &mb, const GemmArgs &a,
                          int grid, cudaStream_t s)
{
    cudaError_t e = set_attr<CM, CN, BK>();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = config(CM * CN, grid, Shape<BK>::SMEM_BYTES, s, attr);
    return cudaLaunchKernelEx(&cfg, k_gemm_bf16<CM, CN, BK>, ma, mb, a);
}

int gemm_max_ctas(int cluster, int bk, int num_sms)
{
    const int key = cluster * 100 + bk;
    switch (key) {
    case 164: return max_ctas<1, 1, 64>(num_sms);
    case 264: return max_ctas<2, 1, 64>(num_sms);
    case 464: return max_ctas<2, 2, 64>(num_sms);
    case 132: return max_ctas<1, 1, 32>(num_sms);
    case 232: return max_ctas<2, 1, 32>(num_sms);
    case 432: return max_ctas<2, 2, 32>(num_sms);
    default: return 0;
    }
}

cudaError_t launch_gemm_bf16(const void *map_a, const void *map_b, const GemmArgs &a,
                             int cluster, int bk, int grid, cudaStream_t s)
{
    CUtensorMap ma, mb;
    memcpy(&ma, map_a, sizeof ma);
    memcpy(&mb, map_b, sizeof mb);
    switch (cluster * 100 + bk) {
    case 164: return launch<1, 1, 64>(ma, mb, a, grid, s);
    case 264: return launch<2, 1, 64>(ma, mb, a, grid, s);
    case 464: return launch<2, 2, 64>(ma, mb, a, grid, s);
    case 132: return launch<1, 1, 32>(ma, mb, a, grid, s);
    case 232: return launch<2, 1, 32>(ma, mb, a, grid, s);
    case 432: return launch<2, 2, 32>(ma, mb, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gw
