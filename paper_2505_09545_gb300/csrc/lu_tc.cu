// Tensor-core trailing update of the FP32 LU on GB300: A22 -= A21 U12 with tcgen05 (TF32 inputs,
// FP32 accumulation in tensor memory), operands staged by TMA.
//
// Complex -> real embedding. With L = A21 (m x nb complex) and U = U12 (nb x m complex), column-major
// interleaved storage makes the trailing block a real (2m) x m matrix C (row 2i+c = component c of
// complex row i). Then
//     C -= Lx * Ur,   Lx = (2m) x (2nb) real, rows 2i: [Lr, -Li, ...], rows 2i+1: [Li, Lr, ...],
//                     Ur = (2nb) x m real = U12 seen as reals (column j = [Ur0, Ui0, Ur1, Ui1, ...]),
// a single real GEMM with M' = 2m, N = m, K' = 2nb and exactly the complex flop count 8 m^2 nb.
// Both operands are K-major: Lx is written K-major by a small preparation kernel, Ur is read directly
// from the matrix (each column of U12 is contiguous in K'). C is updated in place by the epilogue.
//
// Precision modes:  TF32_REFINE: one product per step (TF32 inputs).
//                   FP32:        three products hi*hi + hi*lo + lo*hi of TF32 hi/lo splits (x = hi + lo,
//                                hi = x rounded to TF32), which carries ~21 significant bits.
//
// Kernel structure (persistent, one CTA per SM, 192 threads):
//   warp 0: TMA producer (one elected lane) -> smem ring of STAGES stages (mbarrier full/empty),
//   warp 1: TMEM allocation + MMA issuer (one lane): 128 x BN accumulator per tile, two accumulators
//           (double buffered) so the epilogue of tile t overlaps the main loop of tile t+1,
//   warps 2-5: epilogue: tcgen05.ld of the accumulator (each warp its 32-lane quarter), C -= acc with
//           coalesced column accesses (32 consecutive rows per warp per column).
// Every wait is bounded (~2 s): on timeout the kernel records GDM_ERR_TIMEOUT, drains what it issued,
// frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

#include "gdm_internal.cuh"

namespace {

constexpr int BM = 128;          // rows of the real embedding per tile (UMMA M)
constexpr int BK = 32;           // K' floats per stage = 128 bytes = one 128B swizzle row
constexpr int NTHREADS = 192;

template <int BN, int SPLIT> struct Cfg {
    static constexpr int NP = (SPLIT == 3) ? 2 : 1;  // operand planes per stage (hi[, lo])
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int STAGE_BYTES = NP * (A_BYTES + B_BYTES);
    // operand stages and C staging buffers share the 227 KB: the TF32 update (48 KB stages) takes four
    // stages and two C buffers unless GDM_TC_STAGES3 selects three and four at build time
#ifdef GDM_TC_STAGES3
    static constexpr int STAGES = 3;
    static constexpr int NCB = (SPLIT == 3) ? 2 : 4;
#else
    static constexpr int STAGES = (SPLIT == 3) ? 3 : 4;
    static constexpr int NCB = 2;
#endif
    static constexpr int TMEM_COLS = 2 * BN;
    static constexpr int CB_BYTES = BM * 32 * 4;
    static constexpr int LOOK = NCB / 2;                      // C chunks loaded ahead
    static constexpr int SMEM = STAGES * STAGE_BYTES + NCB * CB_BYTES + 1024 /*alignment*/ + 512 /*barriers*/;
    // instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = BN
    static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(BM >> 4) << 24);
    // the same descriptor with the MMA's N set to n_cols (a multiple of 32 up to BN): narrow column tiles
    // (the last one of a GEMM whose N is not a multiple of BN, or a GEMM narrower than BN) run only the
    // columns that exist
    static __device__ __forceinline__ uint32_t idesc_n(int n_cols) {
        return (IDESC & ~(0x3Fu << 17)) | ((uint32_t)(n_cols >> 3) << 17);
    }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of the given parity. Returns false if the CTA is aborting or after
// ~2 s (then records GDM_ERR_TIMEOUT and raises the CTA's abort flag).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *gflags) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > 2000000000ull) {
                gdm_dev_error(gflags, GDM_ERR_TIMEOUT, 2);
                *abort_flag = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)map),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row core groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void umma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

struct TileMap {
    int num_m, num_n, group;
    // 32-column chunks of column tile nt that hold columns < N (tiles are bn wide)
    __device__ __forceinline__ int chunks(int nt, int N, int bn) const {
        const int left = N - nt * bn;
        return left >= bn ? bn / 32 : (left + 31) / 32;
    }
    __device__ __forceinline__ void get(int t, int &m, int &n) const {
        // groups of `group` column tiles; inside a group the row tile varies slowest across the
        // group's columns so that concurrently running CTAs share operand tiles in L2
        int per_group = num_m * group;
        int g = t / per_group;
        int idx = t - g * per_group;
        int gn = min(group, num_n - g * group);
        n = g * group + idx % gn;
        m = idx / gn;
    }
};

template <int BN, int SPLIT>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_update(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                const __grid_constant__ CUtensorMap tmC, int cx0, int cy0, int M, int N, int K, int bx0, int by0,
                int *gflags) {
    using CF = Cfg<BN, SPLIT>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(base + CF::STAGES * CF::STAGE_BYTES);
    uint64_t *full = bars;                       // [STAGES]
    uint64_t *empty = bars + CF::STAGES;         // [STAGES]
    uint64_t *tfull = bars + 2 * CF::STAGES;     // [2]
    uint64_t *tempty = tfull + 2;                // [2]
    uint64_t *drain = tempty + 2;                // [1]
    uint64_t *cbar = drain + 1;                  // [NCB] C chunk loads
    float *cbuf = (float *)(base + CF::STAGES * CF::STAGE_BYTES + 512);  // NCB x (32 cols x 128 rows)
    uint32_t *tmem_slot = (uint32_t *)(cbar + CF::NCB);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (K + BK - 1) / BK;
    TileMap tm{(M + BM - 1) / BM, (N + BN - 1) / BN, 8};
    const int ntiles = tm.num_m * tm.num_n;

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(drain, 1);
        for (int b = 0; b < CF::NCB; b++) mbar_init(&cbar[b], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)CF::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;  // stages issued and not yet known complete (for the drain on abort)
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                int mt, nt;
                tm.get(t, mt, nt);
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, gflags)) break;
                    unsigned char *st = base + s * CF::STAGE_BYTES;
                    mbar_expect_tx(&full[s], CF::STAGE_BYTES);
                    tma_load_2d(st, &tmA0, kc * BK, mt * BM, &full[s]);
                    tma_load_2d(st + CF::A_BYTES, &tmB0, bx0 + kc * BK, by0 + nt * BN, &full[s]);
                    if (SPLIT == 3) {
                        tma_load_2d(st + CF::A_BYTES + CF::B_BYTES, &tmA1, kc * BK, mt * BM, &full[s]);
                        tma_load_2d(st + 2 * CF::A_BYTES + CF::B_BYTES, &tmB1, bx0 + kc * BK, by0 + nt * BN, &full[s]);
                    }
                    issued++;
                    if (++s == CF::STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            if (*abort_flag) {
                // let the copies already issued land before the CTA's shared memory goes away
                int s2 = s, ph2 = ph;
                for (int i = 0; i < CF::STAGES && i < issued; i++) {
                    if (--s2 < 0) {
                        s2 = CF::STAGES - 1;
                        ph2 ^= 1;
                    }
                    uint64_t t0 = gtimer();
                    while (!mbar_try_wait(&full[s2], ph2) && gtimer() - t0 < 2000000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int lt = 0;
            bool issued_any = false;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, lt++) {
                const int b = lt & 1;
                const uint32_t tph = (lt >> 1) & 1;
                if (!mbar_wait(&tempty[b], tph ^ 1, abort_flag, gflags)) break;
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(b * BN);
                int mt_i, nt_i;
                tm.get(t, mt_i, nt_i);
                const uint32_t idesc = CF::idesc_n(32 * tm.chunks(nt_i, N, BN));
                bool ok = true;
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&full[s], ph, abort_flag, gflags)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(base + s * CF::STAGE_BYTES);
                    const uint64_t a0 = desc_sw128(sa);
                    const uint64_t b0 = desc_sw128(sa + CF::A_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / 8; k++) {
                        // advance 8 TF32 = 32 bytes along K inside the swizzled row: +2 in the 16-B address field
                        const uint64_t ko = (uint64_t)(2 * k);
                        umma_tf32(dt, a0 + ko, b0 + ko, idesc, (kc | k) ? 1u : 0u);
                        if (SPLIT == 3) {
                            const uint64_t a1 = desc_sw128(sa + CF::A_BYTES + CF::B_BYTES);
                            const uint64_t b1 = desc_sw128(sa + 2 * CF::A_BYTES + CF::B_BYTES);
                            umma_tf32(dt, a0 + ko, b1 + ko, idesc, 1u);
                            umma_tf32(dt, a1 + ko, b0 + ko, idesc, 1u);
                        }
                    }
                    issued_any = true;
                    umma_commit(&empty[s]);
                    if (++s == CF::STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit(&tfull[b]);
            }
            if (issued_any) {
                // all MMAs of this CTA complete before tensor memory is released
                umma_commit(drain);
                uint64_t t0 = gtimer();
                while (!mbar_try_wait(drain, 0) && gtimer() - t0 < 2000000000ull) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5 cover the four 32-lane quarters of tensor memory.
        // C streams through shared memory in 128 x 32 chunks: TMA loads run LOOK chunks ahead into a ring of
        // NCB buffers, every thread subtracts its accumulator row, one thread issues the TMA store.
        const int q = warp & 3;
        const int et = threadIdx.x - 64;  // 0..127
        const bool leader = (et == 0);
        // Chunks are numbered over the valid 32-column chunks of this CTA's tiles only (a narrow tile has
        // fewer than BN/32); g indexes that sequence, and the loads run LOOK chunks ahead on a cursor.
        auto tile_chunks = [&](int lt2, int &mt, int &nt) {
            tm.get(blockIdx.x + lt2 * gridDim.x, mt, nt);
            return tm.chunks(nt, N, BN);
        };
        int total = 0;
        for (int t2 = blockIdx.x; t2 < ntiles; t2 += gridDim.x) {
            int mt, nt;
            tm.get(t2, mt, nt);
            total += tm.chunks(nt, N, BN);
        }
        int ld_lt = 0, ld_ch = 0;  // load cursor: tile (local index) and chunk of the next chunk to load
        auto issue_load = [&](int g) {
            int mt, nt;
            const int nch = tile_chunks(ld_lt, mt, nt);
            const int b = g % CF::NCB;
            mbar_expect_tx(&cbar[b], CF::CB_BYTES);
            tma_load_2d(cbuf + (size_t)b * (CF::CB_BYTES / 4), &tmC, cx0 + mt * BM, cy0 + nt * BN + ld_ch * 32,
                        &cbar[b]);
            if (++ld_ch == nch) {
                ld_ch = 0;
                ld_lt++;
            }
        };
        if (leader)
            for (int g = 0; g < CF::LOOK && g < total; g++) issue_load(g);
        int g = 0;  // valid chunks consumed so far
        const int row = q * 32 + lane;
        // Only the leader waits on mbarriers; it publishes each outcome in dec[] (two parity slots) before a
        // named barrier of the four epilogue warps, so all of them take the same branch (no divergent exit).
        volatile int *dec = (volatile int *)(abort_flag + 1);
        int dc = 0;
        auto agree = [&](bool leader_ok) -> bool {
            if (leader) dec[dc & 1] = leader_ok ? 1 : 0;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            bool r = dec[dc & 1] != 0;
            dc++;
            return r;
        };
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, lt++) {
            const int b = lt & 1;
            const uint32_t tph = (lt >> 1) & 1;
            bool ok = true;
            if (leader) ok = mbar_wait(&tfull[b], tph, abort_flag, gflags);
            if (!agree(ok)) break;
            tc_fence_after();
            bool alive = true;
            int mt_c, nt_c;
            const int nch = tile_chunks(lt, mt_c, nt_c);
#pragma unroll 1
            for (int ch = 0; ch < nch; ch++, g++) {
                const int cb = g % CF::NCB;
                ok = true;
                if (leader) {
                    if (g + CF::LOOK < total) {
                        // the buffer's previous chunk (g + LOOK - NCB) must have been read out by its store
                        bulk_wait_read<CF::NCB - CF::LOOK - 1>();
                        issue_load(g + CF::LOOK);
                    }
                    ok = mbar_wait(&cbar[cb], (uint32_t)((g / CF::NCB) & 1), abort_flag, gflags);
                }
                float v[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + ch * 32), v);
                if (!agree(ok)) {
                    alive = false;
                    break;
                }
                float *buf = cbuf + (size_t)cb * (CF::CB_BYTES / 4);
#pragma unroll
                for (int j = 0; j < 32; j++) buf[j * BM + row] -= v[j];
                fence_proxy_async_smem();
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (leader) {
                    tma_store_2d(&tmC, buf, cx0 + mt_c * BM, cy0 + nt_c * BN + ch * 32);
                    bulk_commit();
                }
            }
            if (!alive) break;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (leader) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)CF::TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- grouped update of a batch
// k_tc_update (TF32, one product, 128 x 256 tiles) over the tiles of every problem of one lock-step launch
// of the grouped LU: tile t belongs to the problem whose range of the prefix sum holds it, and its operands
// come through that problem's tensor maps: A = the TF32 embedding of L that the panel kernel wrote (GluItem
// lxp / lxt), B = U read straight from the matrix (rounded to TF32 by the interchange and solve kernel),
// C = the matrix. The maps clip only at the matrix edge, so real rows of a tile at or beyond its region's
// mlim are loaded and stored back unchanged (no other tile of the launch touches them).
struct GDec {
    const GluMaps *m;
    GluTile t;
};
__device__ __forceinline__ GDec glu_decode(const GluItem *__restrict__ items, const GluMaps *__restrict__ maps,
                                           const int *__restrict__ prefix, int na, int kind, int64_t b0, int64_t c0,
                                           int nbo, int t) {
    int lo = 0, hi = na;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&prefix[mid]) <= t) lo = mid;
        else hi = mid;
    }
    GDec d;
    d.m = &maps[lo];
    d.t = glu_tile(kind, items[lo].n, b0, c0, nbo, t - __ldg(&prefix[lo]));
    return d;
}
// the tensor maps were written by the host before the launch; order those writes before the copies that
// read the descriptor
__device__ __forceinline__ void tmap_acquire(const void *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)map) : "memory");
}

// stages of operands, C chunk buffers and C chunks loaded ahead: the K = 32 updates (two K chunks per tile)
// mostly stream C and keep four of eight C buffers loading; the K = nbo updates split the room between three
// operand stages and four C buffers, two of them loading (deeper look-ahead, six of eight and three of five,
// measured no faster)
template <int ST, int NC, int LK> struct GCfg {
    static constexpr int STAGES = ST, NCB = NC, LOOK = LK;  // LOOK C chunks loaded ahead, LOOK < NCB
    static_assert(LK >= 1 && LK < NC, "C look-ahead");
    static constexpr int A_BYTES = BM * BK * 4, B_BYTES = 256 * BK * 4, STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int CB_BYTES = BM * 32 * 4, TMEM_COLS = 512;
    static constexpr int SMEM = ST * STAGE_BYTES + NC * CB_BYTES + 1024 + 512;
    static __device__ __forceinline__ uint32_t idesc_n(int n_cols) { return Cfg<256, 1>::idesc_n(n_cols); }
};
using GCfgPanel = GCfg<2, 8, 4>;
using GCfgTrail = GCfg<3, 4, 2>;

template <class CF>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_glu_gemm(const GluItem *__restrict__ items, const GluMaps *__restrict__ maps, const int *__restrict__ prefix,
               int na, int ntiles, int kind, int64_t b0, int64_t c0, int nbo, int *gflags) {
    constexpr int BN = 256;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(base + CF::STAGES * CF::STAGE_BYTES);
    uint64_t *full = bars;                       // [STAGES]
    uint64_t *empty = bars + CF::STAGES;         // [STAGES]
    uint64_t *tfull = bars + 2 * CF::STAGES;     // [2]
    uint64_t *tempty = tfull + 2;                // [2]
    uint64_t *drain = tempty + 2;                // [1]
    uint64_t *cbar = drain + 1;                  // [NCB] C chunk loads
    float *cbuf = (float *)(base + CF::STAGES * CF::STAGE_BYTES + 512);  // NCB x (32 cols x 128 rows)
    uint32_t *tmem_slot = (uint32_t *)(cbar + CF::NCB);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = kind == GLU_PANEL ? 64 : 2 * nbo;
    const int nk = K / BK;
    const int64_t org = kind == GLU_PANEL ? c0 + 32 : b0 + nbo;  // origin (row and column) of the regions
    const int kx0 = (int)(2 * (kind == GLU_PANEL ? c0 : b0));     // B: real rows of U
    const int cx0 = (int)(2 * org), cy0 = (int)org;
    // A: the panel's column pair range and the first row below it, in the embedding of the block's L
    const int ax0 = kind == GLU_PANEL ? (int)(2 * (c0 - b0)) : 0, ay0 = (int)(2 * (org - b0));

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(drain, 1);
        for (int b = 0; b < CF::NCB; b++) mbar_init(&cbar[b], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)CF::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            const GluMaps *last = nullptr;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const GDec d = glu_decode(items, maps, prefix, na, kind, b0, c0, nbo, t);
                const CUtensorMap *am = (const CUtensorMap *)&d.m->lx;
                const CUtensorMap *bm = (const CUtensorMap *)&d.m->b;
                if (d.m != last) {
                    tmap_acquire(am);
                    tmap_acquire(bm);
                    last = d.m;
                }
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, gflags)) break;
                    unsigned char *st = base + s * CF::STAGE_BYTES;
                    mbar_expect_tx(&full[s], CF::STAGE_BYTES);
                    tma_load_2d(st, am, ax0 + kc * BK, ay0 + d.t.mt * BM, &full[s]);
                    tma_load_2d(st + CF::A_BYTES, bm, kx0 + kc * BK, cy0 + d.t.col0, &full[s]);
                    issued++;
                    if (++s == CF::STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            if (*abort_flag) {
                // let the copies already issued land before the CTA's shared memory goes away
                int s2 = s, ph2 = ph;
                for (int i = 0; i < CF::STAGES && i < issued; i++) {
                    if (--s2 < 0) {
                        s2 = CF::STAGES - 1;
                        ph2 ^= 1;
                    }
                    uint64_t t0 = gtimer();
                    while (!mbar_try_wait(&full[s2], ph2) && gtimer() - t0 < 2000000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int lt = 0;
            bool issued_any = false;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, lt++) {
                const int b = lt & 1;
                const uint32_t tph = (lt >> 1) & 1;
                if (!mbar_wait(&tempty[b], tph ^ 1, abort_flag, gflags)) break;
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(b * BN);
                const GDec d = glu_decode(items, maps, prefix, na, kind, b0, c0, nbo, t);
                const uint32_t idesc = CF::idesc_n(32 * ((d.t.ncols + 31) / 32));
                bool ok = true;
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&full[s], ph, abort_flag, gflags)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(base + s * CF::STAGE_BYTES);
                    const uint64_t a0 = desc_sw128(sa);
                    const uint64_t bd = desc_sw128(sa + CF::A_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / 8; k++) {
                        const uint64_t ko = (uint64_t)(2 * k);
                        umma_tf32(dt, a0 + ko, bd + ko, idesc, (kc | k) ? 1u : 0u);
                    }
                    issued_any = true;
                    umma_commit(&empty[s]);
                    if (++s == CF::STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit(&tfull[b]);
            }
            if (issued_any) {
                umma_commit(drain);
                uint64_t t0 = gtimer();
                while (!mbar_try_wait(drain, 0) && gtimer() - t0 < 2000000000ull) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, as in k_tc_update; the C loads run LOOK chunks ahead on a
        // cursor that walks this CTA's tiles and their valid 32-column chunks
        const int q = warp & 3;
        const int et = threadIdx.x - 64;  // 0..127
        const bool leader = (et == 0);
        int ld_t = blockIdx.x, ld_ch = 0;
        GDec ld_d;
        const GluMaps *last = nullptr;
        if (leader && ld_t < ntiles) ld_d = glu_decode(items, maps, prefix, na, kind, b0, c0, nbo, ld_t);
        auto issue_load = [&](int g) {
            const int b = g % CF::NCB;
            const CUtensorMap *cm = (const CUtensorMap *)&ld_d.m->c;
            if (ld_d.m != last) {
                tmap_acquire(cm);
                last = ld_d.m;
            }
            mbar_expect_tx(&cbar[b], CF::CB_BYTES);
            tma_load_2d(cbuf + (size_t)b * (CF::CB_BYTES / 4), cm, cx0 + ld_d.t.mt * BM, cy0 + ld_d.t.col0 + ld_ch * 32,
                        &cbar[b]);
            if (++ld_ch == (ld_d.t.ncols + 31) / 32) {
                ld_ch = 0;
                ld_t += gridDim.x;
                if (ld_t < ntiles) ld_d = glu_decode(items, maps, prefix, na, kind, b0, c0, nbo, ld_t);
            }
        };
        if (leader)
            for (int g = 0; g < CF::LOOK && ld_t < ntiles; g++) issue_load(g);
        int g = 0;
        const int row = q * 32 + lane;
        volatile int *dec = (volatile int *)(abort_flag + 1);
        int dc = 0;
        auto agree = [&](bool leader_ok) -> bool {
            if (leader) dec[dc & 1] = leader_ok ? 1 : 0;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            bool r = dec[dc & 1] != 0;
            dc++;
            return r;
        };
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, lt++) {
            const int b = lt & 1;
            const uint32_t tph = (lt >> 1) & 1;
            bool ok = true;
            if (leader) ok = mbar_wait(&tfull[b], tph, abort_flag, gflags);
            if (!agree(ok)) break;
            tc_fence_after();
            bool alive = true;
            const GDec d = glu_decode(items, maps, prefix, na, kind, b0, c0, nbo, t);
            const int nch = (d.t.ncols + 31) / 32;
            const bool live_row = d.t.mt * BM + row < d.t.mlim;
#pragma unroll 1
            for (int ch = 0; ch < nch; ch++, g++) {
                const int cb = g % CF::NCB;
                ok = true;
                if (leader) {
                    if (ld_t < ntiles) {
                        // the buffer's previous chunk must have been read out by its store
                        bulk_wait_read<CF::NCB - CF::LOOK - 1>();
                        issue_load(g + CF::LOOK);
                    }
                    ok = mbar_wait(&cbar[cb], (uint32_t)((g / CF::NCB) & 1), abort_flag, gflags);
                }
                float v[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + ch * 32), v);
                if (!agree(ok)) {
                    alive = false;
                    break;
                }
                float *buf = cbuf + (size_t)cb * (CF::CB_BYTES / 4);
                if (live_row) {
#pragma unroll
                    for (int j = 0; j < 32; j++) buf[j * BM + row] -= v[j];
                }
                fence_proxy_async_smem();
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (leader) {
                    tma_store_2d((const CUtensorMap *)&d.m->c, buf, cx0 + d.t.mt * BM, cy0 + d.t.col0 + ch * 32);
                    bulk_commit();
                }
            }
            if (!alive) break;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (leader) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)CF::TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- CTA-pair variant (TF32, one product)
// The same update with 256-row tiles on a CTA pair (a cluster of two CTAs on two SMs): tcgen05.mma with
// cta_group::2 multiplies a 256 x 32 A slab (128 rows in each CTA's shared memory) by a 32 x N B slab whose
// columns are split between the two CTAs (N/2 each), into 128 x N accumulators in each CTA's tensor memory.
// Each CTA fetches only its own half of A and of B, so per pair a B tile crosses L2 once where two
// independent CTAs fetched it twice: operand traffic per flop falls by a third, and the 32 KB stages (against
// 48 KB) leave room for five of them and four C chunk buffers (two C loads in flight ahead of the epilogue,
// whose read-modify-write of C otherwise waits on one HBM round trip per 32-column chunk).
//   leader CTA (rank 0): warp 0 TMA producer (its halves), warp 1 MMA issuer for the pair, warps 2-5 epilogue
//     of rows 0..127 of each tile;
//   peer CTA (rank 1):   warp 0 TMA producer (its halves), warps 2-5 epilogue of rows 128..255.
// Both producers complete their copies on the leader's stage barrier (which expects both CTAs' bytes); the
// MMA commits release the stage in both CTAs and signal both CTAs' epilogues; both epilogues release an
// accumulator on the leader's barrier. Every wait is bounded as in k_tc_update.
constexpr int PBM = 256;         // rows of the real embedding per pair tile (MMA M)
constexpr int PBN = 256;         // columns per pair tile (MMA N); each CTA holds PBN / 2 of B
constexpr int P_STAGES = 5;
constexpr int P_NCB = 4;          // C chunk buffers: loads run P_NCB / 2 chunks ahead of the subtraction
constexpr int P_A_BYTES = 128 * BK * 4;
constexpr int P_B_BYTES = (PBN / 2) * BK * 4;
constexpr int P_STAGE_BYTES = P_A_BYTES + P_B_BYTES;
constexpr int P_CB_BYTES = 128 * 32 * 4;
constexpr int P_SMEM = P_STAGES * P_STAGE_BYTES + P_NCB * P_CB_BYTES + 1024 + 512;
constexpr int P_TMEM_COLS = 2 * PBN;
// D = F32, A = B = TF32, both K-major, M = 256, N = PBN
constexpr uint32_t P_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(PBN >> 3) << 17) |
                             ((uint32_t)(PBM >> 4) << 24);
// kind::f16 with BF16 A and B (format 1), D = F32
constexpr uint32_t P_IDESC_BF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PBN >> 3) << 17) |
                                  ((uint32_t)(PBM >> 4) << 24);
template <bool BF16> __device__ __forceinline__ uint32_t p_idesc_n(int n_cols) {
    return ((BF16 ? P_IDESC_BF16 : P_IDESC) & ~(0x3Fu << 17)) | ((uint32_t)(n_cols >> 3) << 17);
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// 2D tile load into this CTA's shared memory, completing on an mbarrier that may sit in the peer CTA
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y, uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}
__device__ __forceinline__ void umma_tf32_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
// arrive once on the mbarrier at this shared-memory offset in both CTAs of the pair when the pair's MMAs
// issued so far have completed
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// BF16: the same tiles with BF16 operands (64 elements = 128 bytes per stage row, MMA K = 16), for the
// GDM_BF16_REFINE trailing update; the operands are BF16 copies prepared by k_prep_lx_bf16 / k_u_to_bf16.
// MODE 0: C -= A B; MODE 1: C = -A B and MODE 2: C = -A B rounded to TF32 (nearest), both without loading C
// (the U12 product, U12 = -negM A12, written over the block's rows of the trailing columns).
template <bool BF16, int MODE = 0>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    k_tc_update_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmC, int cx0, int cy0, int M, int N, int K, int bx0, int by0,
                     int *gflags) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(base + P_STAGES * P_STAGE_BYTES);
    uint64_t *full = bars;                     // [P_STAGES] (leader's are used)
    uint64_t *empty = bars + P_STAGES;         // [P_STAGES]
    uint64_t *tfull = bars + 2 * P_STAGES;     // [2]
    uint64_t *tempty = tfull + 2;              // [2]   (leader's are used)
    uint64_t *drain = tempty + 2;              // [1]
    uint64_t *cbar = drain + 1;                // [P_NCB]
    float *cbuf = (float *)(base + P_STAGES * P_STAGE_BYTES + 512);
    uint32_t *tmem_slot = (uint32_t *)(cbar + P_NCB);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    constexpr int KE = BF16 ? 2 * BK : BK;  // K elements per stage (128 bytes per row)
    const int nk = (K + KE - 1) / KE;
    TileMap tm{(M + PBM - 1) / PBM, (N + PBN - 1) / PBN, 8};
    const int ntiles = tm.num_m * tm.num_n;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P_STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);  // four epilogue warps in each CTA
        }
        mbar_init(drain, 1);
        for (int b = 0; b < P_NCB; b++) mbar_init(&cbar[b], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)P_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    // both CTAs' barriers are initialised before any copy or arrival crosses to the other CTA
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs): this CTA's 128 rows of A and PBN/2 columns of B
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            for (int t = pair; t < ntiles && !*abort_flag; t += npairs) {
                int mt, nt;
                tm.get(t, mt, nt);
                const int ncol = 32 * tm.chunks(nt, N, PBN);  // MMA N of this tile
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, gflags)) break;
                    unsigned char *st = base + s * P_STAGE_BYTES;
                    const uint32_t fb = mapa_rank(smem_u32(&full[s]), 0);
                    if (leader) mbar_expect_tx(&full[s], 2 * P_STAGE_BYTES);
                    tma_load_2d_pair(st, &tmA, kc * KE, mt * PBM + (int)rank * 128, fb);
                    tma_load_2d_pair(st + P_A_BYTES, &tmB, bx0 + kc * KE, by0 + nt * PBN + (int)rank * (ncol / 2), fb);
                    issued++;
                    if (++s == P_STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            if (*abort_flag && leader) {
                // let the copies already expected land before the pair's shared memory goes away
                int s2 = s, ph2 = ph;
                for (int i = 0; i < P_STAGES && i < issued; i++) {
                    if (--s2 < 0) {
                        s2 = P_STAGES - 1;
                        ph2 ^= 1;
                    }
                    uint64_t t0 = gtimer();
                    while (!mbar_try_wait(&full[s2], ph2) && gtimer() - t0 < 2000000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (leader only)
        if (lane == 0 && leader) {
            int s = 0;
            uint32_t ph = 0;
            int lt = 0;
            bool issued_any = false;
            for (int t = pair; t < ntiles && !*abort_flag; t += npairs, lt++) {
                const int b = lt & 1;
                const uint32_t tph = (lt >> 1) & 1;
                if (!mbar_wait(&tempty[b], tph ^ 1, abort_flag, gflags)) break;
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(b * PBN);
                int mt_i, nt_i;
                tm.get(t, mt_i, nt_i);
                const uint32_t idesc = p_idesc_n<BF16>(32 * tm.chunks(nt_i, N, PBN));
                bool ok = true;
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&full[s], ph, abort_flag, gflags)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(base + s * P_STAGE_BYTES);
                    const uint64_t a0 = desc_sw128(sa);
                    const uint64_t b0 = desc_sw128(sa + P_A_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / 8; k++) {
                        // 32 bytes along K per MMA (8 TF32 or 16 BF16): +2 in the 16-byte address field
                        const uint64_t ko = (uint64_t)(2 * k);
                        if (BF16) umma_bf16_pair(dt, a0 + ko, b0 + ko, idesc, (kc | k) ? 1u : 0u);
                        else umma_tf32_pair(dt, a0 + ko, b0 + ko, idesc, (kc | k) ? 1u : 0u);
                    }
                    issued_any = true;
                    umma_commit_pair(&empty[s]);
                    if (++s == P_STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit_pair(&tfull[b]);
            }
            // all MMAs of the pair complete before tensor memory is released (the commit reaches both CTAs)
            if (issued_any) umma_commit_pair(drain);
            else mbar_arrive_cluster(mapa_rank(smem_u32(drain), 1)), mbar_arrive(drain);
        }
        if (lane == 0) {
            uint64_t t0 = gtimer();
            while (!mbar_try_wait(drain, 0) && gtimer() - t0 < 2000000000ull) {
            }
        }
    } else {
        // ---------------- epilogue (both CTAs): rows rank*128 .. +128 of each tile, as in k_tc_update
        const int q = warp & 3;
        const int et = threadIdx.x - 64;  // 0..127
        const bool eleader = (et == 0);
        const uint32_t tempty_leader0 = mapa_rank(smem_u32(&tempty[0]), 0);
        const uint32_t tempty_leader1 = mapa_rank(smem_u32(&tempty[1]), 0);
        // valid 32-column chunks of a tile for this CTA: none when its 128 rows lie beyond M
        auto tile_chunks = [&](int lt2, int &mt, int &nt) {
            tm.get(pair + lt2 * npairs, mt, nt);
            if (mt * PBM + (int)rank * 128 >= M) return 0;
            return tm.chunks(nt, N, PBN);
        };
        int total = 0;
        for (int lt2 = 0; pair + lt2 * npairs < ntiles; lt2++) {
            int mt, nt;
            total += tile_chunks(lt2, mt, nt);
        }
        int ld_lt = 0, ld_ch = 0;
        auto issue_load = [&](int g) {
            int mt, nt;
            int nch = tile_chunks(ld_lt, mt, nt);
            while (nch == 0) nch = tile_chunks(++ld_lt, mt, nt);
            const int b = g % P_NCB;
            mbar_expect_tx(&cbar[b], P_CB_BYTES);
            tma_load_2d(cbuf + (size_t)b * (P_CB_BYTES / 4), &tmC, cx0 + mt * PBM + (int)rank * 128,
                        cy0 + nt * PBN + ld_ch * 32, &cbar[b]);
            if (++ld_ch == nch) {
                ld_ch = 0;
                ld_lt++;
            }
        };
        if (MODE == 0 && eleader)
            for (int g = 0; g < P_NCB / 2 && g < total; g++) issue_load(g);
        int g = 0;
        const int row = q * 32 + lane;
        volatile int *dec = (volatile int *)(abort_flag + 1);
        int dc = 0;
        auto agree = [&](bool leader_ok) -> bool {
            if (eleader) dec[dc & 1] = leader_ok ? 1 : 0;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            bool r = dec[dc & 1] != 0;
            dc++;
            return r;
        };
        int lt = 0;
        for (int t = pair; t < ntiles; t += npairs, lt++) {
            const int b = lt & 1;
            const uint32_t tph = (lt >> 1) & 1;
            bool ok = true;
            if (eleader) ok = mbar_wait(&tfull[b], tph, abort_flag, gflags);
            if (!agree(ok)) break;
            tc_fence_after();
            bool alive = true;
            int mt_c, nt_c;
            const int nch = tile_chunks(lt, mt_c, nt_c);
#pragma unroll 1
            for (int ch = 0; ch < nch; ch++, g++) {
                const int cb = g % P_NCB;
                ok = true;
                if (eleader) {
                    if (MODE == 0) {
                        if (g + P_NCB / 2 < total) {
                            bulk_wait_read<P_NCB - P_NCB / 2 - 1>();
                            issue_load(g + P_NCB / 2);
                        }
                        ok = mbar_wait(&cbar[cb], (uint32_t)((g / P_NCB) & 1), abort_flag, gflags);
                    } else {
                        // the store that last used buffer cb (chunk g - P_NCB) has read it
                        bulk_wait_read<P_NCB - 1>();
                    }
                }
                float v[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * PBN + ch * 32), v);
                if (!agree(ok)) {
                    alive = false;
                    break;
                }
                float *buf = cbuf + (size_t)cb * (P_CB_BYTES / 4);
                if (MODE == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j++) buf[j * 128 + row] -= v[j];
                } else if (MODE == 1) {
#pragma unroll
                    for (int j = 0; j < 32; j++) buf[j * 128 + row] = -v[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 32; j++) buf[j * 128 + row] = tf32_round(-v[j]);
                }
                fence_proxy_async_smem();
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (eleader) {
                    tma_store_2d(&tmC, buf, cx0 + mt_c * PBM + (int)rank * 128, cy0 + nt_c * PBN + ch * 32);
                    bulk_commit();
                }
            }
            if (!alive) break;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(b ? tempty_leader1 : tempty_leader0);
        }
        if (eleader) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    // no CTA of the pair leaves while the other may still signal its barriers or share its tensor memory
    cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)P_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- operand preparation

// Lx[(2i+c) * K' + 2k + c'] from L = A21 (complex column-major at L, ld lda), rows i < m, cols k < nb.
// SPLIT = 3 writes the TF32 hi part to Lx and the remainder to Llo.
// SPLIT = 1 with Ut: the z = 1 slice of the grid also writes U12 (complex nb x n_cols at U, ld ldu) as a
// K-major real plane Ut[j][2nb] rounded to TF32, so that both operands of a single-product update are rounded
// to nearest rather than truncated by the tensor core.
template <int SPLIT>
__global__ void k_prep_lx(const float2 *__restrict__ L, int64_t lda, int m, int nb, float *__restrict__ Lx,
                          float *__restrict__ Llo, const float2 *__restrict__ U = nullptr, int64_t ldu = 0,
                          int n_cols = 0, float *__restrict__ Ut = nullptr) {
    if (blockIdx.z == 1) {
        const int64_t total = (int64_t)nb * n_cols;
        const int64_t stride = (int64_t)gridDim.x * gridDim.y * blockDim.x;
        for (int64_t e = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x; e < total;
             e += stride) {
            const int j = (int)(e / nb), k = (int)(e % nb);
            const float2 v = U[(int64_t)j * ldu + k];
            *(float2 *)(Ut + (int64_t)j * 2 * nb + 2 * k) = make_float2(tf32_round(v.x), tf32_round(v.y));
        }
        return;
    }
    __shared__ float2 tile[32][33];
    const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int kk = ty; kk < 32; kk += 8) {
        int i = i0 + tx, k = k0 + kk;
        float2 v = make_float2(0.f, 0.f);
        if (i < m && k < nb) v = L[(int64_t)k * lda + i];
        tile[kk][tx] = v;
    }
    __syncthreads();
    const int K2 = 2 * nb;
    for (int ii = ty; ii < 32; ii += 8) {
        int i = i0 + ii, k = k0 + tx;
        if (i >= m || k >= nb) continue;
        float2 l = tile[tx][ii];
        float2 r0 = make_float2(l.x, -l.y), r1 = make_float2(l.y, l.x);
        float2 *o0 = (float2 *)(Lx + (int64_t)(2 * i) * K2 + 2 * k);
        float2 *o1 = (float2 *)(Lx + (int64_t)(2 * i + 1) * K2 + 2 * k);
        if (SPLIT == 3) {
            float2 h0 = make_float2(tf32_round(r0.x), tf32_round(r0.y));
            float2 h1 = make_float2(tf32_round(r1.x), tf32_round(r1.y));
            *o0 = h0;
            *o1 = h1;
            *(float2 *)(Llo + (int64_t)(2 * i) * K2 + 2 * k) = make_float2(r0.x - h0.x, r0.y - h0.y);
            *(float2 *)(Llo + (int64_t)(2 * i + 1) * K2 + 2 * k) = make_float2(r1.x - h1.x, r1.y - h1.y);
        } else {
            // rounded to TF32 here (nearest): the tensor core would otherwise drop the low mantissa bits, a
            // truncation whose bias accumulates over the K sums of the update
            *o0 = make_float2(tf32_round(r0.x), tf32_round(r0.y));
            *o1 = make_float2(tf32_round(r1.x), tf32_round(r1.y));
        }
    }
}

// U12 (complex nb x m at U, ld lda) -> K-major real planes Uhi/Ulo [j][2nb]
__global__ void k_split_u(const float2 *__restrict__ U, int64_t lda, int nb, int m, float *__restrict__ Uhi,
                          float *__restrict__ Ulo) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * m) return;
    int j = (int)(e / nb), k = (int)(e % nb);
    float2 v = U[(int64_t)j * lda + k];
    float2 h = make_float2(tf32_round(v.x), tf32_round(v.y));
    *(float2 *)(Uhi + (int64_t)j * 2 * nb + 2 * k) = h;
    *(float2 *)(Ulo + (int64_t)j * 2 * nb + 2 * k) = make_float2(v.x - h.x, v.y - h.y);
}

// BF16 operands of the GDM_BF16_REFINE trailing update, rounded to nearest even:
// Lb[(2i+c) * K' + 2k + c'] as Lx above, and Ub[j * K' + 2k + c] = U12 column j seen as reals (K-major)
__global__ void k_prep_lx_bf16(const float2 *__restrict__ L, int64_t lda, int m, int nb, __nv_bfloat16 *__restrict__ Lb) {
    __shared__ float2 tile[32][33];
    const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int kk = ty; kk < 32; kk += 8) {
        int i = i0 + tx, k = k0 + kk;
        float2 v = make_float2(0.f, 0.f);
        if (i < m && k < nb) v = L[(int64_t)k * lda + i];
        tile[kk][tx] = v;
    }
    __syncthreads();
    const int K2 = 2 * nb;
    for (int ii = ty; ii < 32; ii += 8) {
        int i = i0 + ii, k = k0 + tx;
        if (i >= m || k >= nb) continue;
        const float2 l = tile[tx][ii];
        *(__nv_bfloat162 *)(Lb + (int64_t)(2 * i) * K2 + 2 * k) = __floats2bfloat162_rn(l.x, -l.y);
        *(__nv_bfloat162 *)(Lb + (int64_t)(2 * i + 1) * K2 + 2 * k) = __floats2bfloat162_rn(l.y, l.x);
    }
}

__global__ void k_u_to_bf16(const float2 *__restrict__ U, int64_t lda, int nb, int m, __nv_bfloat16 *__restrict__ Ub) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)nb * m) return;
    int j = (int)(e / nb), k = (int)(e % nb);
    const float2 v = U[(int64_t)j * lda + k];
    *(__nv_bfloat162 *)(Ub + (int64_t)j * 2 * nb + 2 * k) = __floats2bfloat162_rn(v.x, v.y);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D FP32 tensor map: inner extent `inner` (contiguous), `outer` rows with row pitch `pitch_floats`,
// box 32 x box_rows, 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap *map, const float *gptr, uint64_t inner, uint64_t outer, uint64_t pitch_floats,
              uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch_floats * 4};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)gptr, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 2D BF16 tensor map: inner extent `inner` elements (contiguous), `outer` rows with row pitch `pitch` elements,
// box 64 x box_rows (128-byte rows), 128-byte swizzle, zero fill out of bounds.
bool make_map_bf16(CUtensorMap *map, const __nv_bfloat16 *gptr, uint64_t inner, uint64_t outer, uint64_t pitch,
                   uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch * 2};
    cuuint32_t box[2] = {(cuuint32_t)(2 * BK), box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)gptr, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 2D FP32 tensor map for the C chunks: inner extent `inner` (real rows), `outer` columns with pitch
// pitch_floats, box 128 rows x 32 columns, no swizzle (rows contiguous in shared memory).
bool make_map_c(CUtensorMap *map, const float *gptr, uint64_t inner, uint64_t outer, uint64_t pitch_floats) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch_floats * 4};
    cuuint32_t box[2] = {(cuuint32_t)BM, 32};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)gptr, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, int SPLIT>
gdm_status launch_update(gdm_ctx *ctx, const CUtensorMap &a0, const CUtensorMap &a1, const CUtensorMap &b0,
                         const CUtensorMap &b1, const CUtensorMap &cm, int cx0, int cy0, int M, int N, int K, int bx0,
                         int by0) {
    using CF = Cfg<BN, SPLIT>;
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_update<BN, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               CF::SMEM));
        attr = true;
    }
    int ntiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int grid = ntiles < ctx->sm_count ? ntiles : ctx->sm_count;
    k_tc_update<BN, SPLIT><<<grid, NTHREADS, CF::SMEM, ctx->stream>>>(a0, a1, b0, b1, cm, cx0, cy0, M, N, K, bx0,
                                                                       by0, ctx->dflags);
    GDM_LAUNCHED(ctx, "tc_update");
    return GDM_OK;
}

// CTA pairs that fit on the GPU at once with the pair kernel's shared memory (a persistent grid larger than
// that would leave some pairs waiting for others to finish)
template <bool BF16> int max_pairs(gdm_ctx *ctx) {
    static int cached = -1;
    if (cached < 0) {
        // the occupancy query needs the kernel's shared-memory limit raised first
        if (cudaFuncSetAttribute(k_tc_update_pair<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(ctx->sm_count & ~1));
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = P_SMEM;
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = 2;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (void *)k_tc_update_pair<BF16>, &cfg) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 0;
        }
        cached = n;
    }
    return cached;
}

template <bool BF16, int MODE = 0>
gdm_status launch_update_pair(gdm_ctx *ctx, const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &cm,
                              int cx0, int cy0, int M, int N, int K, int bx0, int by0) {
    const int np = max_pairs<BF16>(ctx);  // raises the kernel's shared-memory limit on first use
    if (np < 1) return GDM_ERR_UNSUPPORTED;
    if (MODE != 0) {
        static bool attr = false;
        if (!attr) {
            GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_update_pair<BF16, MODE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM));
            attr = true;
        }
    }
    const int ntiles = ((M + PBM - 1) / PBM) * ((N + PBN - 1) / PBN);
    const int pairs = ntiles < np ? ntiles : np;
    k_tc_update_pair<BF16, MODE><<<2 * pairs, NTHREADS, P_SMEM, ctx->stream>>>(a, b, cm, cx0, cy0, M, N, K, bx0,
                                                                                by0, ctx->dflags);
    GDM_LAUNCHED(ctx, BF16 ? "tc_update_pair_bf16" : "tc_update_pair");
    return GDM_OK;
}

}  // namespace

size_t gdm_tc_workspace_bytes(int64_t n, int64_t nb, gdm_precision prec) {
    if (prec == GDM_FP64) return 0;
    size_t lx = (size_t)2 * n * 2 * nb * sizeof(float);  // Lx: (2m) x (2nb)
    size_t u = (size_t)n * 2 * nb * sizeof(float);       // one U plane: m x (2nb)
    // TF32: Lx and a rounded copy of U12; BF16_REFINE: BF16 copies of both (12 m nb bytes) fit in the same space
    return prec == GDM_FP32 ? 2 * lx + 2 * u + 4096 : lx + u + 4096;
}

// C[r0 : r0+Mc, c0 : c0+Nc] -= L[0 : Mc, 0 : Kc] U[u_r0 : u_r0+Kc, u_c0 : u_c0+Nc] with complex64 operands in
// column-major storage (C with ldc, L with ldl, U with ldu); C may alias L or U only as disjoint blocks.
// The C chunks are clipped to the sub-block through the tensor-map extents (rows < r0+Mc, columns
// < c0+Nc), so columns and rows outside it are never written. prof = 1 records the launch as the
// factorisation's dominant kernel (gdm_profile_enable). Single-product (TF32) updates read both operands
// rounded to TF32 (nearest): Lx by its preparation, U through a rounded copy unless u_is_tf32 says that U
// holds TF32 values already. out_mode 1 writes C = -L U and 2 writes C = -L U rounded to TF32 (nearest),
// neither reading C: only the single-product update on CTA pairs does this; GDM_ERR_UNSUPPORTED (nothing
// launched) where that kernel does not apply.
gdm_status gdm_tc_update_ext(gdm_ctx *ctx, gdm_precision prec, float2 *C, int64_t ldc, int64_t r0, int64_t c0,
                             const float2 *L, int64_t ldl, const float2 *U, int64_t ldu, int64_t u_r0, int64_t u_c0,
                             int64_t Mc, int64_t Nc, int64_t Kc, void *ws, size_t ws_bytes, int prof,
                             int u_is_tf32, int out_mode) {
    if (prec == GDM_FP64) return GDM_ERR_UNSUPPORTED;
    if (Mc <= 0 || Nc <= 0 || Kc <= 0) return GDM_OK;
    if (getenv("GDM_TC_DISABLE")) return GDM_ERR_UNSUPPORTED;
    if (((uintptr_t)C & 15) || (ldc & 1) || (r0 & 1) || ((uintptr_t)U & 15) || (ldu & 1) || (u_r0 & 1))
        return GDM_ERR_UNSUPPORTED;
    const int split = (prec == GDM_FP32) ? 3 : 1;
    const int M = (int)(2 * Mc), N = (int)Nc, K = (int)(2 * Kc);
    if (out_mode != 0 && (split != 1 || (prec == GDM_BF16_REFINE && prof) || M < PBM || N < 2 * PBN ||
                          getenv("GDM_TC_SINGLE") || max_pairs<false>(ctx) < 1))
        return GDM_ERR_UNSUPPORTED;
    if (prec == GDM_BF16_REFINE && prof && M >= PBM && N >= 2 * PBN && !getenv("GDM_TC_SINGLE") &&
        max_pairs<true>(ctx) >= 1) {
        // the trailing update in BF16 on CTA pairs; BF16 copies of the embedded L panel and of U12
        ScratchCarver sb(ws);
        __nv_bfloat16 *Lb = sb.take<__nv_bfloat16>((size_t)M * K);
        __nv_bfloat16 *Ub = sb.take<__nv_bfloat16>((size_t)N * K);
        if (sb.off > ws_bytes) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "tensor-core workspace too small");
        dim3 pg((unsigned)((Mc + 31) / 32), (unsigned)((Kc + 31) / 32));
        k_prep_lx_bf16<<<pg, 256, 0, ctx->stream>>>(L, ldl, (int)Mc, (int)Kc, Lb);
        GDM_LAUNCHED(ctx, "prep_lx_bf16");
        const int64_t cnt = Kc * Nc;
        k_u_to_bf16<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(U + u_c0 * ldu + u_r0, ldu, (int)Kc,
                                                                            (int)Nc, Ub);
        GDM_LAUNCHED(ctx, "u_to_bf16");
        CUtensorMap ta, tb, tcm;
        if (!(make_map_bf16(&ta, Lb, K, M, K, 128) && make_map_bf16(&tb, Ub, K, N, K, PBN / 2) &&
              make_map_c(&tcm, (const float *)C, (uint64_t)(2 * (r0 + Mc)), (uint64_t)(c0 + Nc), (uint64_t)2 * ldc)))
            return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        int slot = -1;
        const double fl = 8.0 * (double)Mc * (double)Nc * (double)Kc;
        const double by = 16.0 * (double)Mc * Nc + 2.0 * ((double)M * K + (double)N * K);
        GDM_TRY(gdm_prof_begin(ctx, &slot));
        GDM_TRY(launch_update_pair<true>(ctx, ta, tb, tcm, (int)(2 * r0), (int)c0, M, N, K, 0, 0));
        return gdm_prof_end(ctx, slot, fl, by);
    }
    // every other update (and BF16_REFINE's in-block and U12 updates) in TF32
    ScratchCarver sc(ws);
    float *Lx = sc.take<float>((size_t)M * K);
    float *Llo = split == 3 ? sc.take<float>((size_t)M * K) : nullptr;
    float *Uhi = split == 3 ? sc.take<float>((size_t)N * K) : nullptr;
    float *Ulo = split == 3 ? sc.take<float>((size_t)N * K) : nullptr;
    if (sc.off > ws_bytes) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "tensor-core workspace too small");
    dim3 pg((unsigned)((Mc + 31) / 32), (unsigned)((Kc + 31) / 32));
    if (split == 3) {
        k_prep_lx<3><<<pg, 256, 0, ctx->stream>>>(L, ldl, (int)Mc, (int)Kc, Lx, Llo);
        GDM_LAUNCHED(ctx, "prep_lx");
        int64_t cnt = Kc * Nc;
        k_split_u<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(U + u_c0 * ldu + u_r0, ldu, (int)Kc, (int)Nc,
                                                                          Uhi, Ulo);
        GDM_LAUNCHED(ctx, "split_u");
    }
    // single product: a TF32-rounded K-major copy of U12 next to Lx, made by the same launch
    float *Ut = nullptr;
    if (split == 1) {
        if (!u_is_tf32 && !getenv("GDM_TC_TRUNCATE")) {
            Ut = sc.take<float>((size_t)N * K);
            if (sc.off > ws_bytes) return gdm_fail(ctx, GDM_ERR_INVALID_ARG, "tensor-core workspace too small");
        }
        dim3 pg1(pg.x, pg.y, Ut ? 2 : 1);
        k_prep_lx<1><<<pg1, 256, 0, ctx->stream>>>(L, ldl, (int)Mc, (int)Kc, Lx, nullptr, U + u_c0 * ldu + u_r0, ldu,
                                                   (int)Nc, Ut);
        GDM_LAUNCHED(ctx, "prep_lx");
    }
    CUtensorMap ta0, ta1, tb0, tb1, tc;
    bool ok = make_map(&ta0, Lx, K, M, K, BM) &&
              make_map_c(&tc, (const float *)C, (uint64_t)(2 * (r0 + Mc)), (uint64_t)(c0 + Nc), (uint64_t)2 * ldc);
    int slot = -1;
    double fl = 8.0 * (double)Mc * (double)Nc * (double)Kc;
    double by = 16.0 * (double)Mc * Nc + 4.0 * ((double)M * K + (double)N * K) * (split == 3 ? 2 : 1);
    if (split == 3) {
        ok = ok && make_map(&ta1, Llo, K, M, K, BM) && make_map(&tb0, Uhi, K, N, K, 128) &&
             make_map(&tb1, Ulo, K, N, K, 128);
        if (!ok) return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        if (prof) GDM_TRY(gdm_prof_begin(ctx, &slot));
        GDM_TRY(launch_update<128, 3>(ctx, ta0, ta1, tb0, tb1, tc, (int)(2 * r0), (int)c0, M, N, K, 0, 0));
    } else {
        // U straight from its storage: real rows [2 u_r0, 2 u_r0 + K) of columns [u_c0, u_c0 + Nc) (zero beyond)
        // 256-row tiles on CTA pairs (each CTA loads 128 columns of U), unless the update has fewer rows
        // (narrow GEMMs, the in-block updates of at most 256 columns, keep the single-CTA tiles, which do
        // better there)
        const bool pair = M >= PBM && N >= 2 * PBN && !getenv("GDM_TC_SINGLE");
        if (Ut) {
            ok = ok && make_map(&tb0, Ut, K, N, K, pair ? PBN / 2 : 256);
        } else {
            ok = ok && make_map(&tb0, (const float *)U, (uint64_t)2 * ldu, (uint64_t)(u_c0 + Nc), (uint64_t)2 * ldu,
                                pair ? PBN / 2 : 256);
        }
        if (!ok) return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        if (prof) GDM_TRY(gdm_prof_begin(ctx, &slot));
        gdm_status st = GDM_ERR_UNSUPPORTED;
        if (pair) {
            const int bx = Ut ? 0 : (int)(2 * u_r0), by = Ut ? 0 : (int)u_c0;
            if (out_mode == 1)
                st = launch_update_pair<false, 1>(ctx, ta0, tb0, tc, (int)(2 * r0), (int)c0, M, N, K, bx, by);
            else if (out_mode == 2)
                st = launch_update_pair<false, 2>(ctx, ta0, tb0, tc, (int)(2 * r0), (int)c0, M, N, K, bx, by);
            else
                st = launch_update_pair<false>(ctx, ta0, tb0, tc, (int)(2 * r0), (int)c0, M, N, K, bx, by);
        }
        if (st == GDM_ERR_UNSUPPORTED && out_mode != 0) return GDM_ERR_UNSUPPORTED;
        if (st == GDM_ERR_UNSUPPORTED) {
            if (pair) {
                ok = Ut ? make_map(&tb0, Ut, K, N, K, 256)
                        : make_map(&tb0, (const float *)U, (uint64_t)2 * ldu, (uint64_t)(u_c0 + Nc), (uint64_t)2 * ldu,
                                   256);
                if (!ok) return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
            }
            st = Ut ? launch_update<256, 1>(ctx, ta0, ta0, tb0, tb0, tc, (int)(2 * r0), (int)c0, M, N, K, 0, 0)
                    : launch_update<256, 1>(ctx, ta0, ta0, tb0, tb0, tc, (int)(2 * r0), (int)c0, M, N, K,
                                            (int)(2 * u_r0), (int)u_c0);
        }
        GDM_TRY(st);
    }
    if (prof) GDM_TRY(gdm_prof_end(ctx, slot, fl, by));
    return GDM_OK;
}

// General update of a sub-block of the complex64 matrix A (n x n, lda):
//   A[r0 : r0+Mc, c0 : c0+Nc] -= A[r0 : r0+Mc, k0 : k0+Kc] * A[k0 : k0+Kc, c0 : c0+Nc].
gdm_status gdm_tc_update(gdm_ctx *ctx, gdm_precision prec, float2 *A, int64_t lda, int64_t n, int64_t r0, int64_t c0,
                         int64_t k0, int64_t Mc, int64_t Nc, int64_t Kc, void *ws, size_t ws_bytes, int prof) {
    (void)n;
    if ((k0 & 1)) return GDM_ERR_UNSUPPORTED;
    return gdm_tc_update_ext(ctx, prec, A, lda, r0, c0, A + k0 * lda + r0, lda, A, lda, k0, c0, Mc, Nc, Kc, ws,
                             ws_bytes, prof, 0, 0);
}

// A22 -= A21 U12 for the block [b0, b0+nb) of the complex64 matrix A (n x n, lda).
gdm_status gdm_tc_trailing_update(gdm_ctx *ctx, gdm_precision prec, float2 *A, int64_t lda, int64_t n, int64_t b0,
                                  int64_t nb, void *ws, size_t ws_bytes) {
    const int64_t be = b0 + nb, m = n - be;
    if (m < 64) return GDM_ERR_UNSUPPORTED;
    // named range so that profilers can select exactly these launches
    nvtxRangePushA("gdm_trailing_update");
    gdm_status s = gdm_tc_update(ctx, prec, A, lda, n, be, be, b0, m, m, nb, ws, ws_bytes, 1);
    nvtxRangePop();
    return s;
}

// ---------------------------------------------------------------- grouped LU of a batch: maps and launches
bool gdm_glu_encode(const GluItem *items, int n_items, int nbo, GluMaps *maps) {
    for (int i = 0; i < n_items; i++) {
        const GluItem &g = items[i];
        GluMaps &m = maps[i];
        memset(&m, 0, sizeof(m));
        if (g.n <= 32) continue;  // no update reaches a problem of one panel
        if (!(make_map((CUtensorMap *)&m.lx, g.lx, (uint64_t)(2 * nbo), (uint64_t)(2 * g.n), (uint64_t)(2 * nbo),
                       BM) &&
              make_map((CUtensorMap *)&m.b, (const float *)g.A, (uint64_t)(2 * g.n), (uint64_t)g.n,
                       (uint64_t)(2 * g.lda), 256) &&
              make_map_c((CUtensorMap *)&m.c, (const float *)g.A, (uint64_t)(2 * g.n), (uint64_t)g.n,
                         (uint64_t)(2 * g.lda))))
            return false;
    }
    return true;
}

// raises the update kernel's shared-memory limit (once, before any launch is captured into a graph)
gdm_status gdm_glu_gemm_init(gdm_ctx *ctx) {
    static bool attr = false;
    if (!attr) {
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_glu_gemm<GCfgPanel>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               GCfgPanel::SMEM));
        GDM_CUDA_TRY(ctx, cudaFuncSetAttribute(k_glu_gemm<GCfgTrail>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               GCfgTrail::SMEM));
        attr = true;
    }
    return GDM_OK;
}

gdm_status gdm_glu_gemm(gdm_ctx *ctx, const GluItem *items, const GluMaps *maps, const int *prefix, int na,
                        int ntiles, int kind, int64_t b0, int64_t c0, int nbo) {
    if (ntiles <= 0) return GDM_OK;
    GDM_TRY(gdm_glu_gemm_init(ctx));
    const int grid = ntiles < ctx->sm_count ? ntiles : ctx->sm_count;
    if (kind == GLU_PANEL)
        k_glu_gemm<GCfgPanel><<<grid, NTHREADS, GCfgPanel::SMEM, ctx->stream>>>(items, maps, prefix, na, ntiles, kind,
                                                                                b0, c0, nbo, ctx->dflags);
    else
        k_glu_gemm<GCfgTrail><<<grid, NTHREADS, GCfgTrail::SMEM, ctx->stream>>>(items, maps, prefix, na, ntiles, kind,
                                                                                b0, c0, nbo, ctx->dflags);
    GDM_LAUNCHED(ctx, kind == GLU_PANEL ? "glu_gemm_panel" : "glu_gemm_trailing");
    return GDM_OK;
}

// ---------------------------------------------------------------- update from a prepared L embedding
// C[r0 : r0+Mc, c0 : c0+Nc] -= L U (one TF32 product) with the A operand already embedded and rounded to
// TF32 by the panel kernel: real rows 2i and 2i+1 of L's row i at Lx + 2 i lx_pitch, K' = 2 Kc floats each
// (Lx 16-byte aligned, lx_pitch a multiple of 4), and U read straight from its storage (values that are
// TF32 already: rows u_r0 .. u_r0 + Kc of columns u_c0 .. u_c0 + Nc, column-major with ldu). No preparation
// pass: the factorisation's in-block and trailing updates read what the panels and the interchange passes
// wrote. prof = 1 records the launch as the factorisation's dominant kernel.
gdm_status gdm_tc_update_lx(gdm_ctx *ctx, float2 *C, int64_t ldc, int64_t r0, int64_t c0, const float *Lx,
                            int64_t lx_pitch, const float2 *U, int64_t ldu, int64_t u_r0, int64_t u_c0, int64_t Mc,
                            int64_t Nc, int64_t Kc, int prof) {
    if (Mc <= 0 || Nc <= 0 || Kc <= 0) return GDM_OK;
    if (getenv("GDM_TC_DISABLE")) return GDM_ERR_UNSUPPORTED;
    if (((uintptr_t)C & 15) || (ldc & 1) || (r0 & 1) || ((uintptr_t)U & 15) || (ldu & 1) || (u_r0 & 1) ||
        ((uintptr_t)Lx & 15) || (lx_pitch & 3))
        return GDM_ERR_UNSUPPORTED;
    const int M = (int)(2 * Mc), N = (int)Nc, K = (int)(2 * Kc);
    const bool pair = M >= PBM && N >= 2 * PBN && !getenv("GDM_TC_SINGLE");
    CUtensorMap ta, tb, tc;
    if (!(make_map(&ta, Lx, (uint64_t)K, (uint64_t)M, (uint64_t)lx_pitch, BM) &&
          make_map(&tb, (const float *)U, (uint64_t)2 * ldu, (uint64_t)(u_c0 + Nc), (uint64_t)2 * ldu,
                   pair ? PBN / 2 : 256) &&
          make_map_c(&tc, (const float *)C, (uint64_t)(2 * (r0 + Mc)), (uint64_t)(c0 + Nc), (uint64_t)2 * ldc)))
        return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    int slot = -1;
    const double fl = 8.0 * (double)Mc * (double)Nc * (double)Kc;
    const double by = 16.0 * (double)Mc * Nc + 4.0 * ((double)M * K + (double)N * K);
    if (prof) GDM_TRY(gdm_prof_begin(ctx, &slot));
    gdm_status st = GDM_ERR_UNSUPPORTED;
    if (pair)
        st = launch_update_pair<false>(ctx, ta, tb, tc, (int)(2 * r0), (int)c0, M, N, K, (int)(2 * u_r0), (int)u_c0);
    if (st == GDM_ERR_UNSUPPORTED) {
        if (pair && !make_map(&tb, (const float *)U, (uint64_t)2 * ldu, (uint64_t)(u_c0 + Nc), (uint64_t)2 * ldu, 256))
            return gdm_fail(ctx, GDM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        st = launch_update<256, 1>(ctx, ta, ta, tb, tb, tc, (int)(2 * r0), (int)c0, M, N, K, (int)(2 * u_r0),
                                   (int)u_c0);
    }
    GDM_TRY(st);
    if (prof) GDM_TRY(gdm_prof_end(ctx, slot, fl, by));
    return GDM_OK;
}
