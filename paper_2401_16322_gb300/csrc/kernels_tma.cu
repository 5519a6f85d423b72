// Persistent, TMA-fed fused stencil pass (FP32, forward operator) for sm_103a.
//
// Same arithmetic as stage_kernel (kernels_stencil.cu: Eq. 1's operator, Sec. 2.1 stencils,
// Appendix A / Sec. 2.2 free-surface rows, in-register damping, and the
// K / Y / ACC epilogue of every integrator), organised for HBM bandwidth:
//   - one CTA per SM walks the tile work list (tiles b, b + gridDim.x, ...);
//   - warp 8 (one elected lane) is the producer: for each tile it issues TMA tensor loads
//     (cp.async.bulk.tensor) of every operand into one of NST shared-memory stages and
//     arms the stage's "full" mbarrier with the transaction byte count;
//   - warps 0..15 are consumers: they wait on "full", compute the 64 x 16 tile from shared
//     memory (2 consecutive rows per thread, y taps slid in registers), store Y / ACC with
//     coalesced st.global, and arrive on the stage's "empty" mbarrier.
// The TMA boxes (4D tensor maps over x, y, field, vector) start R rows above and 4 columns
// left of the tile (16-byte aligned x); out-of-range elements are filled with zeros by
// the TMA unit, which is exactly the zero extension of Sec. 2.1.
// Every mbarrier wait is bounded (1 s of %globaltimer): on expiry the kernel records an
// error word, drains its own outstanding copies (bounded) and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>
#include <vector>

#include "ewave_internal.cuh"

namespace ewv {

constexpr int TX = 4;                 // staged x halo (>= R, keeps the box start 16-B aligned)
constexpr int NMAP = 12;              // tensor maps per problem and tile height
constexpr int MAX_NST = 5;

// Shared-memory layout of one stage (floats) for tile height BYv; every buffer starts on a
// 128-byte boundary.  HASU = false drops the U buffer (passes without a U operand, e.g. the
// HORK stages) and HASA = false the A buffer (passes without an A operand: the Horner HORK
// passes, the Krylov products), so that more stages or taller tiles fit in shared memory.
template <int R, int BYv, bool HASU = true, bool HASA = true>
struct StageLayout {
    static constexpr int up32(int v) { return (v + 31) / 32 * 32; }   // 128-byte boundary
    static constexpr int SH = BYv + 2 * R;
    static constexpr int SW = BX + 2 * TX;
    static constexpr int U_OFF = 0;                                // u      SH x SW
    static constexpr int WX_OFF = up32(U_OFF + SH * SW);           // w_x    BYv x SW
    static constexpr int WY_OFF = up32(WX_OFF + BYv * SW);         // w_y    SH x BX
    static constexpr int V_OFF = WY_OFF + SH * BX;                 // v      BYv x BX
    static constexpr int C2_OFF = V_OFF + BYv * BX;                // c^2    BYv x BX
    static constexpr int PU_OFF = C2_OFF + BYv * BX;               // U      4 x BYv x BX
    static constexpr int PA_OFF = PU_OFF + (HASU ? 4 * BYv * BX : 0);   // A  4 x BYv x BX
    static constexpr int FLOATS = PA_OFF + (HASA ? 4 * BYv * BX : 0);
    // floats the five field boxes deliver (the padding between buffers is not written)
    static constexpr int BOX_FLOATS = SH * SW + BYv * SW + SH * BX + 2 * BYv * BX;
    static constexpr int BYTES = FLOATS * 4;
    static_assert((U_OFF * 4) % 128 == 0 && (WX_OFF * 4) % 128 == 0 && (WY_OFF * 4) % 128 == 0 &&
                      (V_OFF * 4) % 128 == 0 && (C2_OFF * 4) % 128 == 0 &&
                      (PU_OFF * 4) % 128 == 0 && (PA_OFF * 4) % 128 == 0 && BYTES % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
};

// What the producer resolves once per tile and hands to the consumers with the stage.
struct __align__(16) TileInfo {
    float* Y;
    float* A;
    long long fstr;
    int x0, y0, nx, ny, pitch, pml, fs, src_i, src_j, shot;
    float beta0, inv_pml, idx1, idx2, sig, xs;   // xs: per-problem scale of H X (Krylov)
    const float* btab;       // damping at half-cell distances (ProblemDev::btab)
    int nbtab, pad3;
};

// The consumers read a stage's TileInfo with 16-byte shared loads into registers.
__device__ __forceinline__ TileInfo load_info(const TileInfo* p) {
    static_assert(sizeof(TileInfo) % 16 == 0, "TileInfo must be a whole number of 16-byte words");
    union {
        TileInfo t;
        int4 v[sizeof(TileInfo) / 16];
    } u;
#pragma unroll
    for (int q = 0; q < (int)(sizeof(TileInfo) / 16); ++q) u.v[q] = reinterpret_cast<const int4*>(p)[q];
    return u.t;
}
template <bool kRegs>
__device__ __forceinline__ std::conditional_t<kRegs, TileInfo, const TileInfo&> tile_info(const TileInfo* p) {
    if constexpr (kRegs)
        return load_info(p);
    else
        return *p;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Limit of the pipeline waits (ns).  1 s by default; ewv_debug_set_wait_limit lowers it so
// that a test can make a wait give up on a healthy GPU and check the reported status.  The
// drain after a give-up always waits up to 1 s for the copies still in flight.
__device__ unsigned long long g_tma_wait_limit_ns = 1000000000ull;
constexpr uint64_t kDrainLimitNs = 1000000000ull;

int set_tma_wait_limit_ns(unsigned long long ns) {
    return cudaMemcpyToSymbol(g_tma_wait_limit_ns, &ns, sizeof(ns)) == cudaSuccess ? 0 : -1;
}

// Non-blocking probe of a phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after limit_ns (or 2^26 polls) without the phase completing; with
// limit_ns = 0, false unless the phase has already completed (one non-blocking probe).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (limit_ns == 0) return mbar_test_wait(bar, parity);
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

__constant__ float g_tma_fs[4 * 9 + 3 * 8 + 4 * 8];
constexpr int TFS_UYY = 0, TFS_UY = 36, TFS_DWY = 60;

int upload_tma_tables(const double* fs_uyy, const double* fs_uy, const double* fs_dwy) {
    float f[92];
    for (int i = 0; i < 36; ++i) f[TFS_UYY + i] = (float)fs_uyy[i];
    for (int i = 0; i < 24; ++i) f[TFS_UY + i] = (float)fs_uy[i];
    for (int i = 0; i < 32; ++i) f[TFS_DWY + i] = (float)fs_dwy[i];
    return cudaMemcpyToSymbol(g_tma_fs, f, sizeof(f)) == cudaSuccess ? 0 : -1;
}

template <int R>
__device__ __forceinline__ float stag(int k) {
    if constexpr (R == 4) {
        return k == 0 ? float(1225.0 / 1024.0) : k == 1 ? float(-245.0 / 3072.0)
             : k == 2 ? float(49.0 / 5120.0) : float(-5.0 / 7168.0);
    } else {
        return k == 0 ? float(9.0 / 8.0) : float(-1.0 / 24.0);
    }
}
template <int R>
__device__ __forceinline__ float cent(int k) {
    if constexpr (R == 4) {
        return k == 0 ? float(-205.0 / 72.0) : k == 1 ? float(8.0 / 5.0) : k == 2 ? float(-1.0 / 5.0)
             : k == 3 ? float(8.0 / 315.0) : float(-1.0 / 560.0);
    } else {
        return k == 0 ? float(-5.0 / 2.0) : k == 1 ? float(4.0 / 3.0) : float(-1.0 / 12.0);
    }
}
// Stencil sums as balanced trees (short dependency chains for the issue slots):
// stag_tree = sum_k s_k d[k] over the R staggered differences, cent_tree = c_0 u +
// sum_k c_k p[k-1] over the R symmetric pair sums.
template <int R>
__device__ __forceinline__ float stag_tree(const float (&d)[R]) {
    if constexpr (R == 4)
        return fmaf(stag<4>(0), d[0], stag<4>(1) * d[1]) + fmaf(stag<4>(2), d[2], stag<4>(3) * d[3]);
    else
        return fmaf(stag<R>(0), d[0], stag<R>(1) * d[1]);
}
template <int R>
__device__ __forceinline__ float cent_tree(float u, const float (&p)[R]) {
    if constexpr (R == 4)
        return (fmaf(cent<4>(1), p[0], cent<4>(0) * u) + fmaf(cent<4>(3), p[2], cent<4>(2) * p[1])) +
               cent<4>(4) * p[3];
    else
        return fmaf(cent<R>(1), p[0], cent<R>(0) * u) + cent<R>(2) * p[1];
}

// Two-row arithmetic on packed FP32 pairs (one instruction for both rows of a consumer
// thread; each component rounds exactly as the scalar operation does).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <int R>
__device__ __forceinline__ float2 stag_tree2(const float2 (&d)[R]) {
    if constexpr (R == 4)
        return add2(fma2(f2s(stag<4>(0)), d[0], mul2(f2s(stag<4>(1)), d[1])),
                    fma2(f2s(stag<4>(2)), d[2], mul2(f2s(stag<4>(3)), d[3])));
    else
        return fma2(f2s(stag<R>(0)), d[0], mul2(f2s(stag<R>(1)), d[1]));
}
template <int R>
__device__ __forceinline__ float2 cent_tree2(float2 u, const float2 (&p)[R]) {
    if constexpr (R == 4)
        return add2(add2(fma2(f2s(cent<4>(1)), p[0], mul2(f2s(cent<4>(0)), u)),
                         fma2(f2s(cent<4>(3)), p[2], mul2(f2s(cent<4>(2)), p[1]))),
                    mul2(f2s(cent<4>(4)), p[3]));
    else
        return add2(fma2(f2s(cent<R>(1)), p[0], mul2(f2s(cent<R>(0)), u)), mul2(f2s(cent<R>(2)), p[1]));
}

// beta at 2 d = k half cells from the first ghost line (zero beyond the layer).  Columns and
// rows past the grid edge (ragged tiles, never stored) give k <= 0; the unsigned test sends
// negative k to zero as well, so the table is never read outside its n entries.
__device__ __forceinline__ float btab_at(const float* t, int n, int k) {
    return (unsigned)k < (unsigned)n ? __ldg(t + k) : 0.f;
}

__device__ __forceinline__ float dampf(float beta0, float inv_pml, float d, int pml) {
    if (pml <= 0) return 0.f;
    const float r = 1.f - d * inv_pml;
    return (d <= (float)pml) ? beta0 * r * r : 0.f;
}

// Map of field box `kind` (0 u, 1 w_x, 2 w_y, 3 v, 4 four fields) for vector k.
__device__ __forceinline__ const CUtensorMap* map_of(const CUtensorMap* base, int k, int kind) {
    return base + (k == 0 ? 0 : 5) + kind;
}

// Problem of tile t: the last p with base[p] <= t (base: nprob + 1 prefix sums).
__device__ __forceinline__ int find_problem(const int* __restrict__ base, int nprob, int t) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The tile descriptor the producer hands to the consumers with a stage.
__device__ __forceinline__ void fill_tile_info(TileInfo& ti, const ProblemDev* P, const StageArgs& a, int x0,
                                               int y0) {
    ti.Y = a.y_out >= 0 ? (a.y_out == 0 ? (float*)P->state
                                        : (float*)P->work + (long long)(a.y_out - 1) * P->vec_stride)
                        : nullptr;
    ti.A = a.acc_out >= 0 ? (a.acc_out == 0 ? (float*)P->state
                                            : (float*)P->work + (long long)(a.acc_out - 1) * P->vec_stride)
                          : nullptr;
    ti.fstr = P->field_stride;
    ti.x0 = x0;
    ti.y0 = y0;
    ti.nx = P->nx;
    ti.ny = P->ny;
    ti.pitch = P->pitch;
    ti.pml = P->pml;
    ti.fs = P->fs;
    ti.src_i = P->src_i;
    ti.src_j = P->src_j;
    ti.shot = P->shot;
    ti.btab = P->btab;
    ti.nbtab = P->nbtab;
    ti.beta0 = P->fbeta0;
    ti.inv_pml = P->finv_pml;
    ti.idx1 = P->finv_dx;
    ti.idx2 = P->finv_dx2;
    ti.sig = (a.src_slot >= 0 && P->has_src) ? (float)P->sigma[a.src_slot] : 0.f;
    ti.xs = a.x_scale_slot >= 0 ? (float)P->kry[a.x_scale_slot] : 1.f;
}

// The producer (one elected lane of the last warp): for each tile of this CTA, wait until
// its stage is free, resolve the tile's problem and descriptor, arm the stage's "full"
// barrier with the byte count and issue the TMA loads.  Returns the number of tiles issued.
template <int R, int BYv, int NSTv, int EPI, bool HASU, bool HASA = true>
__device__ __forceinline__ int tma_produce(const ProblemDev* __restrict__ probs, const int* __restrict__ tbase,
                                           int nprob, int ntiles, int mapset, const StageArgs& a, float* smem,
                                           uint64_t* full, uint64_t* empty, TileInfo* info, int* s_err,
                                           uint32_t bytes, uint64_t wait_lim) {
    using L = StageLayout<R, BYv, HASU, HASA>;
    const bool has_u = HASU && a.u >= 0, has_a = HASA && a.a >= 0;
    int issued = 0;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int s = it % NSTv;
        const uint32_t ph = (uint32_t)(it / NSTv) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, wait_lim)) {
            *s_err = 1;
            break;
        }
        const int pid = find_problem(tbase, nprob, tile);
        const ProblemDev* P = probs + pid;
        const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P->tmaps) + mapset * NMAP;
        const int tiles_x = (P->nx + BX - 1) / BX;
        const int lt = tile - __ldg(tbase + pid);
        const int x0 = (lt % tiles_x) * BX, y0 = (lt / tiles_x) * BYv;
        fill_tile_info(info[s], P, a, x0, y0);
        float* st = smem + (size_t)s * L::FLOATS;
        // the arrive below releases the tile info together with the copies
        mbar_expect_tx(&full[s], bytes);
        const int kx = a.x, cx = a.x == 0 ? 0 : a.x - 1;
        tma_load_4d(st + L::U_OFF, map_of(maps, kx, 0), x0 - TX, y0 - R, 0, cx, &full[s]);
        tma_load_4d(st + L::WX_OFF, map_of(maps, kx, 1), x0 - TX, y0, 2, cx, &full[s]);
        tma_load_4d(st + L::WY_OFF, map_of(maps, kx, 2), x0, y0 - R, 3, cx, &full[s]);
        if (EPI < 2) tma_load_4d(st + L::V_OFF, map_of(maps, kx, 3), x0, y0, 1, cx, &full[s]);
        if (EPI != 3) tma_load_2d(st + L::C2_OFF, maps + 10, x0, y0, &full[s]);
        if (has_u)
            tma_load_4d(st + L::PU_OFF, map_of(maps, a.u, 4), x0, y0, 0, a.u == 0 ? 0 : a.u - 1, &full[s]);
        if (has_a)
            tma_load_4d(st + L::PA_OFF, map_of(maps, a.a, 4), x0, y0, 0, a.a == 0 ? 0 : a.a - 1, &full[s]);
        issued = it + 1;
    }
    return issued;
}

// Byte count one stage receives (the "full" barrier's transaction count).
template <int R, int BYv, int EPI, bool HASU, bool HASA = true>
__device__ __forceinline__ uint32_t tma_stage_bytes(const StageArgs& a) {
    using L = StageLayout<R, BYv, HASU, HASA>;
    const bool has_u = HASU && a.u >= 0, has_a = HASA && a.a >= 0;
    // (the leap-frog step, EPI 2, does not read v; the gradient pass, EPI 3, neither v nor c^2)
    return (uint32_t)((L::BOX_FLOATS - (EPI >= 2 ? BYv * BX : 0) - (EPI == 3 ? BYv * BX : 0) +
                       (has_u ? 4 * BYv * BX : 0)) * 4) +
           (has_a ? 4 * BYv * BX * 4 : 0);
}

// After a pipeline wait gave up: the producer waits (bounded) for the last copy issued into
// every stage, so that no TMA write lands after the CTA exits, and the error word is set.
template <int NSTv>
__device__ __forceinline__ void tma_finish(int s_err, int issued, uint64_t* full, int* err) {
    const int tid = threadIdx.x;
    if (s_err) {
        if (issued > 0) {
            for (int it = issued - 1; it >= 0 && it >= issued - NSTv; --it)
                (void)mbar_wait(&full[it % NSTv], (uint32_t)(it / NSTv) & 1u, kDrainLimitNs);
        }
        if (tid == 0) atomicOr(err, 1);
    }
}

// EPI 0: the general epilogue.  EPI 1: the steady-state form of the Faber and HORK passes,
// ck = 1 and cau = cak = cax = 0:  Y = cu U + cx X + ch (H X + sigma),  ACC = ca A + cay Y.
template <int R, int BYv, int NW, int NSTv, int EPI, bool HASU>
__global__ void __launch_bounds__(NW * 32 + 32, 1)
stage_tma_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tbase, int nprob,
                 int ntiles, int mapset, StageArgs a, int* err) {
    using L = StageLayout<R, BYv, HASU>;
    constexpr int NCONS = NW * 32;
    constexpr int TPR = NCONS / BX;             // consumer thread rows
    constexpr int NR = BYv / TPR;               // consecutive rows per consumer thread
    static_assert(NR * TPR == BYv && NR >= 1, "tile rows must split evenly over threads");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // TMA destinations need 128-byte alignment: align the dynamic base explicitly (the
    // launch reserves 1 KB of slack for this).
    float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NSTv];
    __shared__ __align__(8) uint64_t empty[NSTv];
    __shared__ TileInfo info[NSTv];
    __shared__ int s_err;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint64_t wait_lim = g_tma_wait_limit_ns;
    if (tid == 0) {
        for (int s = 0; s < NSTv; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const bool has_u = HASU && a.u >= 0, has_a = a.a >= 0;
    const uint32_t bytes = tma_stage_bytes<R, BYv, EPI, HASU>(a);
    int issued = 0;

    if (warp == NW) {
        // ------------------------------------------------------------ producer
        if (lane == 0)
            issued = tma_produce<R, BYv, NSTv, EPI, HASU>(probs, tbase, nprob, ntiles, mapset, a, smem, full,
                                                          empty, info, &s_err, bytes, wait_lim);
    } else {
        // ------------------------------------------------------------ consumers
        const int tx = tid & (BX - 1);    // x inside the tile
        const int ty = tid / BX;          // rows NR ty .. NR ty + NR - 1
#define cxf a.fcx
#define chf a.fch
#define cuf a.fcu
#define ckf a.fck
#define caf a.fca
#define cauf a.fcau
#define cakf a.fcak
#define cayf a.fcay
#define caxf a.fcax
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % NSTv;
            const uint32_t ph = (uint32_t)(it / NSTv) & 1u;
            if (!mbar_wait(&full[s], ph, wait_lim)) {
                s_err = 1;
                break;
            }
            // The tile descriptor: copied into registers where they are plentiful; read from
            // shared memory field by field by the 20-warp variant (80 registers a thread).
            using TI = std::conditional_t<(NW < 20), const TileInfo, const TileInfo&>;
            TI ti = tile_info<(NW < 20)>(&info[s]);
            const int nx = ti.nx, ny = ti.ny, pml = ti.pml;
            const bool fs = ti.fs != 0;
            const int y0 = ti.y0;
            const long long fstr = ti.fstr;
            const float beta0 = ti.beta0, inv_pml = ti.inv_pml, idx1 = ti.idx1, idx2 = ti.idx2;
            float* Yg = ti.Y;
            float* Ag = ti.A;
            const float* st = smem + (size_t)s * L::FLOATS;
            const float* su = st + L::U_OFF;
            const float* swx = st + L::WX_OFF;
            const float* swy = st + L::WY_OFF;
            const float* sv = st + L::V_OFF;
            const float* sc2 = st + L::C2_OFF;
            const float* spu = st + L::PU_OFF;
            const float* spa = st + L::PA_OFF;
            const int i = ti.x0 + tx;
            const int cxs = tx + TX;                     // staged column of this thread
            float ucol[NR + 2 * R], wcol[NR + 2 * R - 1];
#pragma unroll
            for (int q = 0; q < NR + 2 * R; ++q) ucol[q] = su[(NR * ty + q) * L::SW + cxs];
#pragma unroll
            for (int q = 0; q < NR + 2 * R - 1; ++q) wcol[q] = swy[(NR * ty + q) * BX + tx];
            const float* btab = ti.btab;
            const int nbt = ti.nbtab;
            const float bxn = btab_at(btab, nbt, 2 * min(i + 1, nx - i));
            const float bxh = btab_at(btab, nbt, min(2 * i + 3, 2 * (nx - i) - 1));
            const bool in_x = i < nx;
            const float chx = chf * ti.xs;     // ch xs: K = cx X + ch xs (H X + sigma)
            // EPI 2: one leap-frog step (Sec. 3.1) at a point.  X = level n; the A box holds
            // level n - 1 (u^{n-1} or, in difference form, d^n in field 1, and w^{n-1});
            // level n + 1 goes to Y (u, w_x, w_y) and, in difference form, d^{n+1} to field 1
            // of level n (acc_out), which no thread of this step reads.
            auto leapfrog_point = [&](int ii, int jj, int ptv, float uu, float c2v, float lap, float dws,
                                      float dux, float duy, float bxnv, float bxhv, float bynv, float byhv,
                                      float xwxv, float xwyv) {
                const float dt = (float)a.dt, bsum = bxnv + bynv;
                float rhs = -bxnv * bynv * uu + c2v * (lap * idx2 + dws * idx1);
                if (ii == ti.src_i && jj == ti.src_j) rhs += ti.sig;
                const float* pm = spa + ptv;
                const long long o = (long long)jj * ti.pitch + ii;
                // fast (2-ulp) divisions, as in the 3D step: the step's own error is far larger
                float up;
                if (a.m == 2) {
                    const float hb = 0.5f * bsum * dt;
                    const float dn = __fdividef(pm[BYv * BX] * (1.f - hb) + dt * dt * rhs, 1.f + hb);
                    Ag[fstr + o] = dn;
                    up = uu + dn;
                } else {
                    const float um = pm[0];
                    const float inv_dt2 = 1.f / (dt * dt), inv_2dt = 1.f / (2.f * dt);
                    up = __fdividef((2.f * uu - um) * inv_dt2 + bsum * um * inv_2dt + rhs, inv_dt2 + bsum * inv_2dt);
                }
                float wxp = 0.f, wyp = 0.f;
                if (ii < nx - 1) {
                    const float gx = (bynv - bxhv) * dux * idx1, wm = pm[2 * BYv * BX];
                    wxp = a.m != 1 ? __fdividef((1.f - bxhv * dt) * wm + 2.f * dt * gx, 1.f + bxhv * dt)
                                   : wm + 2.f * dt * (-bxhv * xwxv + gx);
                }
                if (jj < ny - 1) {
                    const float gy = (bxnv - byhv) * duy * idx1, wm = pm[3 * BYv * BX];
                    wyp = a.m != 1 ? __fdividef((1.f - byhv * dt) * wm + 2.f * dt * gy, 1.f + byhv * dt)
                                   : wm + 2.f * dt * (-byhv * xwyv + gy);
                }
                Yg[o] = up;
                Yg[2 * fstr + o] = wxp;
                Yg[3 * fstr + o] = wyp;
            };
            bool paired = false;
            if constexpr (NR == 2 && EPI >= 1) {
                // Both rows of this thread as packed pairs (rows below the free-surface
                // band: the interior stencils apply to both).
                const int ly0 = 2 * ty;
                const int j0 = y0 + ly0, j1 = j0 + 1;
                paired = !(fs && j0 < 4);
                if (paired && in_x && j0 < ny) {
                    const float* urow0 = su + (ly0 + R) * L::SW + cxs;
                    const float* urow1 = urow0 + L::SW;
                    const float* wx0 = swx + ly0 * L::SW + cxs;
                    const float* wx1 = wx0 + L::SW;
                    const float2 uc = f2(ucol[R], ucol[R + 1]);
                    // The pair sums and differences of the taps are packed; the products with
                    // the stencil weights stay scalar (immediate operands, no registers held).
                    // lap = 2 c_0 u + sum_k c_k (x pair sum + y pair sum); the divergence of w
                    // and d_x u, d_y u accumulate their staggered differences the same way.
                    float lap0 = (2.f * cent<R>(0)) * uc.x, lap1 = (2.f * cent<R>(0)) * uc.y;
                    float dw0 = 0.f, dw1 = 0.f, ux0 = 0.f, ux1 = 0.f, uy0 = 0.f, uy1 = 0.f;
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const float2 ap = f2(urow0[k + 1], urow1[k + 1]);
                        const float2 am = f2(urow0[-k - 1], urow1[-k - 1]);
                        const float2 a0 = k == 0 ? uc : f2(urow0[-k], urow1[-k]);
                        const float2 sl = add2(ap, am);
                        const float2 sx = sub2(ap, a0);
                        const float2 sw = sub2(f2(wx0[k], wx1[k]), f2(wx0[-1 - k], wx1[-1 - k]));
                        lap0 = fmaf(cent<R>(k + 1), sl.x + (ucol[R + k + 1] + ucol[R - k - 1]), lap0);
                        lap1 = fmaf(cent<R>(k + 1), sl.y + (ucol[R + k + 2] + ucol[R - k]), lap1);
                        ux0 = fmaf(stag<R>(k), sx.x, ux0);
                        ux1 = fmaf(stag<R>(k), sx.y, ux1);
                        uy0 = fmaf(stag<R>(k), ucol[R - k] - ucol[R + 1 + k], uy0);
                        uy1 = fmaf(stag<R>(k), ucol[R - k + 1] - ucol[R + 2 + k], uy1);
                        dw0 = fmaf(stag<R>(k), sw.x + (wcol[R - 1 - k] - wcol[R + k]), dw0);
                        dw1 = fmaf(stag<R>(k), sw.y + (wcol[R - k] - wcol[R + k + 1]), dw1);
                    }
                    if constexpr (EPI == 3) {
                        // FWI gradient pass: grad += gscale q_v (L u + D w) of X (m = c^2)
                        float* G = (float*)a.grad + (long long)ti.shot * fstr;
                        const long long o0 = (long long)j0 * ti.pitch + i;
                        const float gs = (float)a.gscale;
                        G[o0] += gs * spa[BYv * BX + ly0 * BX + tx] * (lap0 * idx2 + dw0 * idx1);
                        if (j1 < ny) G[o0 + ti.pitch] += gs * spa[BYv * BX + ly0 * BX + BX + tx] * (lap1 * idx2 + dw1 * idx1);
                    } else {
                    const float byn0 = btab_at(btab, nbt, 2 * (fs ? ny - j0 : min(j0 + 1, ny - j0)));
                    const float byn1 = btab_at(btab, nbt, 2 * (fs ? ny - j1 : min(j1 + 1, ny - j1)));
                    const float byh0 = btab_at(btab, nbt, fs ? 2 * (ny - j0) - 1 : min(2 * j0 + 3, 2 * (ny - j0) - 1));
                    const float byh1 = btab_at(btab, nbt, fs ? 2 * (ny - j1) - 1 : min(2 * j1 + 3, 2 * (ny - j1) - 1));
                    const int pt0 = ly0 * BX + tx, pt1 = pt0 + BX;
                    if constexpr (EPI == 2) {
                        leapfrog_point(i, j0, pt0, uc.x, sc2[pt0], lap0, dw0, ux0, uy0, bxn, bxh, byn0, byh0,
                                       wx0[0], wcol[R]);
                        if (j1 < ny)
                            leapfrog_point(i, j1, pt1, uc.y, sc2[pt1], lap1, dw1, ux1, uy1, bxn, bxh, byn1, byh1,
                                           wx1[0], wcol[R + 1]);
                    } else {
                    const float xv0 = sv[pt0], xv1 = sv[pt1];
                    const float xwx0 = wx0[0], xwx1 = wx1[0];
                    const float xwy0 = wcol[R], xwy1 = wcol[R + 1];
                    // H v = -bx by u + c^2 (lap u / dx^2 + div w / dx) - (bx + by) v
                    float hv0 = -bxn * byn0 * uc.x + sc2[pt0] * (lap0 * idx2 + dw0 * idx1) - (bxn + byn0) * xv0;
                    float hv1 = -bxn * byn1 * uc.y + sc2[pt1] * (lap1 * idx2 + dw1 * idx1) - (bxn + byn1) * xv1;
                    if (i == ti.src_i) {
                        if (j0 == ti.src_j) hv0 += ti.sig;
                        if (j1 == ti.src_j) hv1 += ti.sig;
                    }
                    const bool wxin = i < nx - 1;
                    const float hwx0 = wxin ? (byn0 - bxh) * ux0 * idx1 - bxh * xwx0 : 0.f;
                    const float hwx1 = wxin ? (byn1 - bxh) * ux1 * idx1 - bxh * xwx1 : 0.f;
                    const float hwy0 = (j0 < ny - 1) ? (bxn - byh0) * uy0 * idx1 - byh0 * xwy0 : 0.f;
                    const float hwy1 = (j1 < ny - 1) ? (bxn - byh1) * uy1 * idx1 - byh1 * xwy1 : 0.f;
                    const bool row1 = j1 < ny;
                    const long long o0 = (long long)j0 * ti.pitch + i;
                    const float xf0[4] = {uc.x, xv0, xwx0, xwy0}, xf1[4] = {uc.y, xv1, xwx1, xwy1};
                    const float hf0[4] = {xv0, hv0, hwx0, hwy0}, hf1[4] = {xv1, hv1, hwx1, hwy1};
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        float y0v = fmaf(cxf, xf0[f], chx * hf0[f]);
                        float y1v = fmaf(cxf, xf1[f], chx * hf1[f]);
                        if (has_u) {
                            y0v = fmaf(cuf, spu[f * BYv * BX + pt0], y0v);
                            y1v = fmaf(cuf, spu[f * BYv * BX + pt1], y1v);
                        }
                        if ((f == 2 && !wxin) || (f == 3 && j0 >= ny - 1)) y0v = 0.f;
                        if ((f == 2 && !wxin) || (f == 3 && j1 >= ny - 1)) y1v = 0.f;
                        if (Yg) {
                            float* yp = Yg + f * fstr + o0;
                            yp[0] = y0v;
                            if (row1) yp[ti.pitch] = y1v;
                        }
                        if (Ag) {
                            float a0v = cayf * y0v, a1v = cayf * y1v;
                            if (has_a) {
                                a0v = fmaf(cayf, y0v, caf * spa[f * BYv * BX + pt0]);
                                a1v = fmaf(cayf, y1v, caf * spa[f * BYv * BX + pt1]);
                            }
                            float* ap = Ag + f * fstr + o0;
                            ap[0] = a0v;
                            if (row1) ap[ti.pitch] = a1v;
                        }
                    }
                    }   // EPI 1
                    }   // EPI 1, 2
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (paired) break;
                const int ly = NR * ty + r;
                const int j = y0 + ly;
                const float* urow = su + (ly + R) * L::SW + cxs;
                const float* wxrow = swx + ly * L::SW + cxs;
                float px[R], dx[R], dw[R];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    px[k] = urow[k + 1] + urow[-k - 1];
                    dx[k] = urow[1 + k] - urow[-k];
                    dw[k] = wxrow[k] - wxrow[-1 - k];
                }
                const float uxx = cent_tree<R>(ucol[r + R], px);
                const float dux = stag_tree<R>(dx);
                const float dwx = stag_tree<R>(dw);
                float uyy, duy, dwy;
                if (fs && j < 4) {
                    uyy = 0.f;
#pragma unroll
                    for (int q = 0; q < 9; ++q) uyy += g_tma_fs[TFS_UYY + j * 9 + q] * su[(q + R) * L::SW + cxs];
                    dwy = 0.f;
#pragma unroll
                    for (int q = 0; q < 8; ++q) dwy += g_tma_fs[TFS_DWY + j * 8 + q] * swy[(q + R) * BX + tx];
                } else {
                    float py[R], dwv[R];
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        py[k] = ucol[r + R + k + 1] + ucol[r + R - k - 1];
                        dwv[k] = wcol[r + R - 1 - k] - wcol[r + R + k];
                    }
                    uyy = cent_tree<R>(ucol[r + R], py);
                    dwy = stag_tree<R>(dwv);
                }
                if (fs && j < 3) {
                    duy = 0.f;
#pragma unroll
                    for (int q = 0; q < 8; ++q) duy += g_tma_fs[TFS_UY + j * 8 + q] * su[(q + R) * L::SW + cxs];
                } else {
                    float dy[R];
#pragma unroll
                    for (int k = 0; k < R; ++k) dy[k] = ucol[r + R - k] - ucol[r + R + 1 + k];
                    duy = stag_tree<R>(dy);
                }
                if (!in_x || j >= ny) continue;
                const float byn = btab_at(btab, nbt, 2 * (fs ? ny - j : min(j + 1, ny - j)));
                const float byh = btab_at(btab, nbt, fs ? 2 * (ny - j) - 1 : min(2 * j + 3, 2 * (ny - j) - 1));
                const int pt = ly * BX + tx;
                if constexpr (EPI == 3) {
                    float* G = (float*)a.grad + (long long)ti.shot * fstr;
                    G[(long long)j * ti.pitch + i] += (float)a.gscale * spa[BYv * BX + pt] *
                                                      ((uxx + uyy) * idx2 + (dwx + dwy) * idx1);
                    continue;
                }
                if constexpr (EPI == 2) {
                    leapfrog_point(i, j, pt, ucol[r + R], sc2[pt], uxx + uyy, dwx + dwy, dux, duy, bxn, bxh,
                                   byn, byh, wxrow[0], wcol[r + R]);
                    continue;
                }
                const float xu = ucol[r + R], xv = sv[pt], xwx = wxrow[0], xwy = wcol[r + R];
                const float c2 = sc2[pt];
                float hv = -bxn * byn * xu + c2 * ((uxx + uyy) * idx2 + (dwx + dwy) * idx1) - (bxn + byn) * xv;
                if (i == ti.src_i && j == ti.src_j) hv += ti.sig;
                const float hwx = (i < nx - 1) ? (byn - bxh) * dux * idx1 - bxh * xwx : 0.f;
                const float hwy = (j < ny - 1) ? (bxn - byh) * duy * idx1 - byh * xwy : 0.f;
                const float xf[4] = {xu, xv, xwx, xwy};
                const float hf[4] = {xv, hv, hwx, hwy};
                const long long o = (long long)j * ti.pitch + i;
                float* yrow = Yg ? Yg + o : nullptr;
                float* arow = Ag ? Ag + o : nullptr;
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const bool pad = (f == 2 && i >= nx - 1) || (f == 3 && j >= ny - 1);
                    const float uval = has_u ? spu[f * BYv * BX + pt] : 0.f;
                    const float aval = has_a ? spa[f * BYv * BX + pt] : 0.f;
                    const float kf = fmaf(cxf, xf[f], chx * hf[f]);
                    if constexpr (EPI == 1) {
                        const float yf = pad ? 0.f : (has_u ? fmaf(cuf, uval, kf) : kf);
                        if (yrow) yrow[f * fstr] = yf;
                        if (arow) arow[f * fstr] = has_a ? fmaf(cayf, yf, caf * aval) : cayf * yf;
                    } else {
                        const float yf = pad ? 0.f : (cuf * uval + ckf * kf);
                        if (yrow) yrow[f * fstr] = yf;
                        if (arow) arow[f * fstr] = pad ? 0.f : (caf * aval + cauf * uval + cakf * kf + cayf * yf + caxf * xf[f]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    // (issued is non-zero on the producer lane only)
    tma_finish<NSTv>(s_err, issued, full, err);
}

#undef cxf
#undef chf
#undef cuf
#undef ckf
#undef caf
#undef cauf
#undef cakf
#undef cayf
#undef caxf

// ---------------------------------------------------------------- column-pair consumers
// The same pass with every consumer thread on two adjacent columns (x, x + 1) of NR
// consecutive rows: the column pair of a staged row is one 8-byte shared load, and the
// arithmetic runs on packed FP32 pairs (one instruction for both columns).  The y taps of
// both columns slide in registers as pairs; the x taps of a row are the five pairs from
// x - 4 to x + 5, and the taps that straddle two pairs (odd offsets) are formed with scalar
// operations.  Per grid point this issues about a third of the shared loads of the
// one-column form and shares each tile's setup over twice the points.  Rows of the
// free-surface band (Appendix A stencils, top tile only) take a scalar path per point.
__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float2 v, bool both) {
    if (both)
        *reinterpret_cast<float2*>(p) = v;
    else
        p[0] = v.x;
}

// One leap-frog step (Sec. 3.1) at a point of the column-pair form: level n in registers,
// level n - 1 (u^{n-1}, or d^n in field 1 in difference form, and w^{n-1}) from the A stage
// box at pa (fields plane floats apart); level n + 1 (u, w_x, w_y) goes to Y and, in
// difference form, d^{n+1} to field 1 of A.  Same arithmetic as the one-column form.
__device__ __forceinline__ void lf_point(const TileInfo& ti, const StageArgs& a, const float* pa, int plane, int ii,
                                         int jj, float uu, float c2v, float lap, float dws, float dux, float duy,
                                         float bxnv, float bxhv, float bynv, float byhv, float xwxv, float xwyv) {
    const float idx1 = ti.idx1, idx2 = ti.idx2;
    const float dt = (float)a.dt, bsum = bxnv + bynv;
    float rhs = -bxnv * bynv * uu + c2v * (lap * idx2 + dws * idx1);
    if (ii == ti.src_i && jj == ti.src_j) rhs += ti.sig;
    const long long o = (long long)jj * ti.pitch + ii;
    const long long fstr = ti.fstr;
    // fast (2-ulp) divisions, as in the one-column form
    float up;
    if (a.m == 2) {
        const float hb = 0.5f * bsum * dt;
        const float dn = __fdividef(pa[plane] * (1.f - hb) + dt * dt * rhs, 1.f + hb);
        ti.A[fstr + o] = dn;
        up = uu + dn;
    } else {
        const float um = pa[0];
        const float inv_dt2 = 1.f / (dt * dt), inv_2dt = 1.f / (2.f * dt);
        up = __fdividef((2.f * uu - um) * inv_dt2 + bsum * um * inv_2dt + rhs, inv_dt2 + bsum * inv_2dt);
    }
    float wxp = 0.f, wyp = 0.f;
    if (ii < ti.nx - 1) {
        const float gx = (bynv - bxhv) * dux * idx1, wm = pa[2 * plane];
        wxp = a.m != 1 ? __fdividef((1.f - bxhv * dt) * wm + 2.f * dt * gx, 1.f + bxhv * dt)
                       : wm + 2.f * dt * (-bxhv * xwxv + gx);
    }
    if (jj < ti.ny - 1) {
        const float gy = (bxnv - byhv) * duy * idx1, wm = pa[3 * plane];
        wyp = a.m != 1 ? __fdividef((1.f - byhv * dt) * wm + 2.f * dt * gy, 1.f + byhv * dt)
                       : wm + 2.f * dt * (-byhv * xwyv + gy);
    }
    ti.Y[o] = up;
    ti.Y[2 * fstr + o] = wxp;
    ti.Y[3 * fstr + o] = wyp;
}

// One point (tile column tc, tile row lr) from shared memory with the scalar formulas of the
// one-column form, free-surface rows included, and its epilogue.
template <int R, int BYv, int EPI, bool HASU, bool HASA>
__device__ __forceinline__ void tma_point_scalar(const float* st, const TileInfo& ti, const StageArgs& a, int tc,
                                             int lr, bool has_u, bool has_a) {
    using L = StageLayout<R, BYv, HASU, HASA>;
    const int nx = ti.nx, ny = ti.ny;
    const int i = ti.x0 + tc, j = ti.y0 + lr;
    if (i >= nx || j >= ny) return;
    const bool fs = ti.fs != 0;
    const int cs = tc + TX;
    const float* su = st + L::U_OFF;
    const float* swy = st + L::WY_OFF;
    const float* urow = su + (lr + R) * L::SW + cs;
    const float* wxrow = st + L::WX_OFF + lr * L::SW + cs;
    auto ucolv = [&](int q) { return su[(lr + q) * L::SW + cs]; };   // staged row lr + q
    auto wcolv = [&](int q) { return swy[(lr + q) * BX + tc]; };
    float px[R], dx[R], dw[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        px[k] = urow[k + 1] + urow[-k - 1];
        dx[k] = urow[1 + k] - urow[-k];
        dw[k] = wxrow[k] - wxrow[-1 - k];
    }
    const float uc = urow[0];
    const float uxx = cent_tree<R>(uc, px);
    const float dux = stag_tree<R>(dx);
    const float dwx = stag_tree<R>(dw);
    float uyy, duy, dwy;
    if (fs && j < 4) {
        uyy = 0.f;
#pragma unroll
        for (int q = 0; q < 9; ++q) uyy += g_tma_fs[TFS_UYY + j * 9 + q] * su[(q + R) * L::SW + cs];
        dwy = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) dwy += g_tma_fs[TFS_DWY + j * 8 + q] * swy[(q + R) * BX + tc];
    } else {
        float py[R], dwv[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            py[k] = ucolv(R + k + 1) + ucolv(R - k - 1);
            dwv[k] = wcolv(R - 1 - k) - wcolv(R + k);
        }
        uyy = cent_tree<R>(uc, py);
        dwy = stag_tree<R>(dwv);
    }
    if (fs && j < 3) {
        duy = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) duy += g_tma_fs[TFS_UY + j * 8 + q] * su[(q + R) * L::SW + cs];
    } else {
        float dy[R];
#pragma unroll
        for (int k = 0; k < R; ++k) dy[k] = ucolv(R - k) - ucolv(R + 1 + k);
        duy = stag_tree<R>(dy);
    }
    const float* btab = ti.btab;
    const int nbt = ti.nbtab;
    const float bxn = btab_at(btab, nbt, 2 * min(i + 1, nx - i));
    const float bxh = btab_at(btab, nbt, min(2 * i + 3, 2 * (nx - i) - 1));
    const float byn = btab_at(btab, nbt, 2 * (fs ? ny - j : min(j + 1, ny - j)));
    const float byh = btab_at(btab, nbt, fs ? 2 * (ny - j) - 1 : min(2 * j + 3, 2 * (ny - j) - 1));
    const int pt = lr * BX + tc;
    const float* sv = st + L::V_OFF;
    const float* sc2 = st + L::C2_OFF;
    const float* spu = st + L::PU_OFF;
    const float* spa = st + L::PA_OFF;
    if constexpr (EPI == 3) {
        float* G = (float*)a.grad + (long long)ti.shot * ti.fstr;
        G[(long long)j * ti.pitch + i] +=
            (float)a.gscale * spa[BYv * BX + pt] * ((uxx + uyy) * ti.idx2 + (dwx + dwy) * ti.idx1);
        return;
    }
    if constexpr (EPI == 2) {
        lf_point(ti, a, spa + pt, BYv * BX, i, j, uc, sc2[pt], uxx + uyy, dwx + dwy, dux, duy, bxn, bxh, byn,
                 byh, wxrow[0], wcolv(R));
        return;
    }
    const float idx1 = ti.idx1, idx2 = ti.idx2;
    const float xu = uc, xv = sv[pt], xwx = wxrow[0], xwy = wcolv(R);
    float hv = -bxn * byn * xu + sc2[pt] * ((uxx + uyy) * idx2 + (dwx + dwy) * idx1) - (bxn + byn) * xv;
    if (i == ti.src_i && j == ti.src_j) hv += ti.sig;
    const float hwx = (i < nx - 1) ? (byn - bxh) * dux * idx1 - bxh * xwx : 0.f;
    const float hwy = (j < ny - 1) ? (bxn - byh) * duy * idx1 - byh * xwy : 0.f;
    const float xf[4] = {xu, xv, xwx, xwy};
    const float hf[4] = {xv, hv, hwx, hwy};
    const float chx = a.fch * ti.xs;
    const long long o = (long long)j * ti.pitch + i;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool pad = (f == 2 && i >= nx - 1) || (f == 3 && j >= ny - 1);
        const float uval = has_u ? spu[f * BYv * BX + pt] : 0.f;
        const float aval = has_a ? spa[f * BYv * BX + pt] : 0.f;
        const float kf = fmaf(a.fcx, xf[f], chx * hf[f]);
        if constexpr (EPI == 1) {
            const float yf = pad ? 0.f : (has_u ? fmaf(a.fcu, uval, kf) : kf);
            if (ti.Y) ti.Y[f * ti.fstr + o] = yf;
            if (ti.A) ti.A[f * ti.fstr + o] = has_a ? fmaf(a.fcay, yf, a.fca * aval) : a.fcay * yf;
        } else {
            const float yf = pad ? 0.f : (a.fcu * uval + a.fck * kf);
            if (ti.Y) ti.Y[f * ti.fstr + o] = yf;
            if (ti.A)
                ti.A[f * ti.fstr + o] =
                    pad ? 0.f : (a.fca * aval + a.fcau * uval + a.fcak * kf + a.fcay * yf + a.fcax * xf[f]);
        }
    }
}

template <int R, int BYv, int NW, int NSTv, int EPI, bool HASU, bool HASA>
__global__ void __launch_bounds__(NW * 32 + 32, 1)
stage_tma_x2_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tbase, int nprob,
                    int ntiles, int mapset, StageArgs a, int* err) {
    static_assert(EPI <= 3, "EPI 0 / 1: integrator passes, 2: leap-frog step, 3: gradient pass");
    using L = StageLayout<R, BYv, HASU, HASA>;
    constexpr int CPR = BX / 2;                 // consumer threads per tile row
    constexpr int TPR = NW * 32 / CPR;          // thread rows
    constexpr int NR = BYv / TPR;               // consecutive rows per consumer thread
    static_assert(NR * TPR == BYv && NR >= 1, "tile rows must split evenly over threads");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NSTv];
    __shared__ __align__(8) uint64_t empty[NSTv];
    __shared__ TileInfo info[NSTv];
    __shared__ int s_err;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint64_t wait_lim = g_tma_wait_limit_ns;
    if (tid == 0) {
        for (int s = 0; s < NSTv; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool has_u = HASU && a.u >= 0, has_a = HASA && a.a >= 0;
    int issued = 0;
    if (warp == NW) {
        if (lane == 0)
            issued = tma_produce<R, BYv, NSTv, EPI, HASU, HASA>(
                probs, tbase, nprob, ntiles, mapset, a, smem, full, empty, info, &s_err,
                tma_stage_bytes<R, BYv, EPI, HASU, HASA>(a), wait_lim);
    } else {
        const int tx2 = tid % CPR, ty = tid / CPR;
        const int c0 = 2 * tx2;                 // first of the two tile columns
        const int cs = c0 + TX;                 // its staged column (even: 8-byte aligned)
        const int r0 = NR * ty;                 // first tile row of this thread
        const float2 cx2 = f2s(a.fcx), cu2 = f2s(a.fcu), ck2 = f2s(a.fck), ca2 = f2s(a.fca);
        const float2 cay2 = f2s(a.fcay), cau2 = f2s(a.fcau), cak2 = f2s(a.fcak), cax2 = f2s(a.fcax);
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % NSTv;
            const uint32_t ph = (uint32_t)(it / NSTv) & 1u;
            if (!mbar_wait(&full[s], ph, wait_lim)) {
                s_err = 1;
                break;
            }
            const TileInfo ti = load_info(&info[s]);
            const float* st = smem + (size_t)s * L::FLOATS;
            const int nx = ti.nx, ny = ti.ny;
            const int i0 = ti.x0 + c0;
            const int jt = ti.y0 + r0;
            if (i0 < nx && jt < ny) {
                if (ti.fs != 0 && jt < 4) {
                    // free-surface band: one point at a time
#pragma unroll 1
                    for (int r = 0; r < NR; ++r) {
                        tma_point_scalar<R, BYv, EPI, HASU, HASA>(st, ti, a, c0, r0 + r, has_u, has_a);
                        tma_point_scalar<R, BYv, EPI, HASU, HASA>(st, ti, a, c0 + 1, r0 + r, has_u, has_a);
                    }
                } else {
                    const float* su = st + L::U_OFF;
                    const float* swx = st + L::WX_OFF;
                    const float* swy = st + L::WY_OFF;
                    const float* sv = st + L::V_OFF;
                    const float* sc2 = st + L::C2_OFF;
                    const float* spu = st + L::PU_OFF;
                    const float* spa = st + L::PA_OFF;
                    const bool fs = ti.fs != 0;
                    const bool in1 = i0 + 1 < nx;
                    float2 ucol[NR + 2 * R], wcol[NR + 2 * R - 1];
#pragma unroll
                    for (int q = 0; q < NR + 2 * R; ++q) ucol[q] = lds2(su + (r0 + q) * L::SW + cs);
#pragma unroll
                    for (int q = 0; q < NR + 2 * R - 1; ++q) wcol[q] = lds2(swy + (r0 + q) * BX + c0);
                    const float* btab = ti.btab;
                    const int nbt = ti.nbtab;
                    const float2 bxn = f2(btab_at(btab, nbt, 2 * min(i0 + 1, nx - i0)),
                                          btab_at(btab, nbt, 2 * min(i0 + 2, nx - i0 - 1)));
                    const float2 bxh = f2(btab_at(btab, nbt, min(2 * i0 + 3, 2 * (nx - i0) - 1)),
                                          btab_at(btab, nbt, min(2 * i0 + 5, 2 * (nx - i0) - 3)));
                    const float2 nbxh = f2(-bxh.x, -bxh.y);
                    const bool wx0in = i0 < nx - 1, wx1in = i0 + 1 < nx - 1;
                    const float2 idx1 = f2s(ti.idx1), idx2 = f2s(ti.idx2);
                    const float chx = a.fch * ti.xs;
                    const float2 chx2 = f2s(chx);
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int lr = r0 + r, j = jt + r;
                        if (j >= ny) break;
                        // x taps: u and w_x at tile columns c0 - 4 .. c0 + 5 of this row
                        const float* urow = su + (lr + R) * L::SW + cs;
                        const float* wxr = swx + lr * L::SW + cs;
                        const float2 up[5] = {lds2(urow - 4), lds2(urow - 2), ucol[r + R], lds2(urow + 2),
                                              lds2(urow + 4)};
                        const float2 wp[5] = {lds2(wxr - 4), lds2(wxr - 2), lds2(wxr), lds2(wxr + 2),
                                              lds2(wxr + 4)};
                        // scalar tap at column offset d (-4 .. 5) from the first column
                        auto uo = [&](int d) { return ((d + 4) & 1) ? up[(d + 4) >> 1].y : up[(d + 4) >> 1].x; };
                        auto wo = [&](int d) { return ((d + 4) & 1) ? wp[(d + 4) >> 1].y : wp[(d + 4) >> 1].x; };
                        const float2 uc = ucol[r + R];
                        float2 lap = mul2(f2s(2.f * cent<R>(0)), uc);
                        float2 dux = f2s(0.f), duy = f2s(0.f), dw = f2s(0.f);
#pragma unroll
                        for (int k = 0; k < R; ++k) {
                            // Laplacian: x and y pair sums at distance k + 1
                            const int kk = k + 1;
                            const float2 sx = (kk & 1) ? f2(uo(kk) + uo(-kk), uo(kk + 1) + uo(1 - kk))
                                                       : add2(up[(kk + 4) >> 1], up[(4 - kk) >> 1]);
                            const float2 sy = add2(ucol[r + R + kk], ucol[r + R - kk]);
                            lap = fma2(f2s(cent<R>(kk)), add2(sx, sy), lap);
                            // staggered differences: d_x u at x + 1/2, d_y u at y + 1/2,
                            // the divergence of w at the node
                            const float2 dxu = f2(uo(1 + k) - uo(-k), uo(2 + k) - uo(1 - k));
                            dux = fma2(f2s(stag<R>(k)), dxu, dux);
                            duy = fma2(f2s(stag<R>(k)), sub2(ucol[r + R - k], ucol[r + R + 1 + k]), duy);
                            const float2 dxw = f2(wo(k) - wo(-1 - k), wo(1 + k) - wo(-k));
                            const float2 dyw = sub2(wcol[r + R - 1 - k], wcol[r + R + k]);
                            dw = fma2(f2s(stag<R>(k)), add2(dxw, dyw), dw);
                        }
                        const float byn = btab_at(btab, nbt, 2 * (fs ? ny - j : min(j + 1, ny - j)));
                        const float byh =
                            btab_at(btab, nbt, fs ? 2 * (ny - j) - 1 : min(2 * j + 3, 2 * (ny - j) - 1));
                        const int pt = lr * BX + c0;
                        if constexpr (EPI == 3) {
                            // FWI gradient pass: grad += gscale q_v (L u + D w) of X (m = c^2);
                            // q's fields ride in the A box
                            float* G = (float*)a.grad + (long long)ti.shot * ti.fstr +
                                       (long long)j * ti.pitch + i0;
                            const float2 qv = lds2(spa + BYv * BX + pt);
                            const float2 gv = mul2(mul2(f2s((float)a.gscale), qv),
                                                   fma2(lap, f2s(ti.idx2), mul2(dw, f2s(ti.idx1))));
                            if (in1) {
                                float2 g0 = *reinterpret_cast<float2*>(G);
                                *reinterpret_cast<float2*>(G) = add2(g0, gv);
                            } else {
                                G[0] += gv.x;
                            }
                            continue;
                        }
                        if constexpr (EPI == 2) {
                            // one leap-frog step per column of the pair
                            const float2 c2l = lds2(sc2 + pt);
                            lf_point(ti, a, spa + pt, BYv * BX, i0, j, uc.x, c2l.x, lap.x, dw.x, dux.x, duy.x,
                                     bxn.x, bxh.x, byn, byh, wp[2].x, wcol[r + R].x);
                            if (in1)
                                lf_point(ti, a, spa + pt + 1, BYv * BX, i0 + 1, j, uc.y, c2l.y, lap.y, dw.y, dux.y,
                                         duy.y, bxn.y, bxh.y, byn, byh, wp[2].y, wcol[r + R].y);
                            continue;
                        }
                        const float2 xv = lds2(sv + pt), c2 = lds2(sc2 + pt);
                        const float2 xwx = wp[2], xwy = wcol[r + R];
                        // H v = -bx by u + c^2 (lap u / dx^2 + div w / dx) - (bx + by) v
                        const float2 t = fma2(mul2(bxn, f2s(-byn)), uc, mul2(sub2(f2s(-byn), bxn), xv));
                        float2 hv = fma2(c2, fma2(lap, idx2, mul2(dw, idx1)), t);
                        if (j == ti.src_j) {
                            if (i0 == ti.src_i) hv.x += ti.sig;
                            if (i0 + 1 == ti.src_i) hv.y += ti.sig;
                        }
                        float2 hwx = fma2(nbxh, xwx, mul2(mul2(sub2(f2s(byn), bxh), dux), idx1));
                        if (!wx0in) hwx.x = 0.f;
                        if (!wx1in) hwx.y = 0.f;
                        const bool wyin = j < ny - 1;
                        const float2 hwy =
                            wyin ? fma2(f2s(-byh), xwy, mul2(mul2(sub2(bxn, f2s(byh)), duy), idx1)) : f2s(0.f);
                        const float2 xf[4] = {uc, xv, xwx, xwy};
                        const float2 hf[4] = {xv, hv, hwx, hwy};
                        const long long o = (long long)j * ti.pitch + i0;
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            const float2 uval = has_u ? lds2(spu + f * BYv * BX + pt) : f2s(0.f);
                            const float2 aval = has_a ? lds2(spa + f * BYv * BX + pt) : f2s(0.f);
                            const float2 kf = fma2(cx2, xf[f], mul2(chx2, hf[f]));
                            float2 yf, af;
                            if constexpr (EPI == 1) {
                                yf = has_u ? fma2(cu2, uval, kf) : kf;
                            } else {
                                yf = fma2(cu2, uval, mul2(ck2, kf));
                            }
                            if (f == 2) {
                                if (!wx0in) yf.x = 0.f;
                                if (!wx1in) yf.y = 0.f;
                            }
                            if (f == 3 && !wyin) yf = f2s(0.f);
                            if constexpr (EPI == 1) {
                                af = has_a ? fma2(cay2, yf, mul2(ca2, aval)) : mul2(cay2, yf);
                            } else {
                                af = fma2(cax2, xf[f],
                                          fma2(cay2, yf, fma2(cak2, kf, fma2(cau2, uval, mul2(ca2, aval)))));
                                if (f == 2) {
                                    if (!wx0in) af.x = 0.f;
                                    if (!wx1in) af.y = 0.f;
                                }
                                if (f == 3 && !wyin) af = f2s(0.f);
                            }
                            if (ti.Y) st2(ti.Y + f * ti.fstr + o, yf, in1);
                            if (ti.A) st2(ti.A + f * ti.fstr + o, af, in1);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    tma_finish<NSTv>(s_err, issued, full, err);
}

// ---------------------------------------------------------------- transposed pass
// H^T y (the adjoint's passes) with the column-pair consumers.  For y = (y_u, y_v, y_wx,
// y_wy):
//   (H^T y)_u  = -bx by y_v + L (c^2 y_v) - D_x(z_x) - D_y(z_y)      (L symmetric in the interior)
//   (H^T y)_v  = y_u - (bx + by) y_v
//   (H^T y)_wx = -d_x^+(c^2 y_v) - bx^h y_wx                          at (i+1/2, j)
//   (H^T y)_wy = -d_y^+(c^2 y_v) - by^h y_wy                          at (i, j+1/2)
// with z_x = (by - bx^h) y_wx at the half columns and z_y = (bx - by^h) y_wy at the half rows:
// the transposes of the forward's staggered derivatives are the negated staggered
// derivatives of the other grid (zero extension keeps that exact at the edges).  The stage
// carries y_v and c^2 with the 2D halo (their product is formed from shared memory), y_wx
// with the x halo, y_wy with the y halo, y_u and the U / A operands.  The rows whose
// transposed stencils meet the free-surface rows of Appendix A (rows 0..8: the columns of
// those rows) take a scalar path per point that adds the tables' columns.
template <int R, int BYv, bool HASU, bool HASA>
struct TLayout {
    static constexpr int up32(int v) { return (v + 31) / 32 * 32; }
    static constexpr int SH = BYv + 2 * R;
    static constexpr int SW = BX + 2 * TX;
    static constexpr int ZV_OFF = 0;                                 // y_v    SH x SW
    static constexpr int C2_OFF = up32(ZV_OFF + SH * SW);            // c^2    SH x SW
    static constexpr int WX_OFF = up32(C2_OFF + SH * SW);            // y_wx   BYv x SW
    static constexpr int WY_OFF = up32(WX_OFF + BYv * SW);           // y_wy   SH x BX
    static constexpr int YU_OFF = WY_OFF + SH * BX;                  // y_u    BYv x BX
    static constexpr int PU_OFF = YU_OFF + BYv * BX;                 // U      4 x BYv x BX
    static constexpr int PA_OFF = PU_OFF + (HASU ? 4 * BYv * BX : 0);   // A   4 x BYv x BX
    static constexpr int FLOATS = PA_OFF + (HASA ? 4 * BYv * BX : 0);
    static constexpr int BOX_FLOATS = 2 * SH * SW + BYv * SW + SH * BX + BYv * BX;
    static constexpr int BYTES = FLOATS * 4;
    static_assert((C2_OFF * 4) % 128 == 0 && (WX_OFF * 4) % 128 == 0 && (WY_OFF * 4) % 128 == 0 &&
                      (YU_OFF * 4) % 128 == 0 && (PU_OFF * 4) % 128 == 0 && (PA_OFF * 4) % 128 == 0 &&
                      BYTES % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
};

template <int R, int BYv, int NSTv, bool HASU, bool HASA>
__device__ __forceinline__ int tma_produce_t(const ProblemDev* __restrict__ probs, const int* __restrict__ tbase,
                                             int nprob, int ntiles, int mapset, const StageArgs& a, float* smem,
                                             uint64_t* full, uint64_t* empty, TileInfo* info, int* s_err,
                                             uint64_t wait_lim) {
    using L = TLayout<R, BYv, HASU, HASA>;
    const bool has_u = HASU && a.u >= 0, has_a = HASA && a.a >= 0;
    const uint32_t bytes = (uint32_t)(L::BOX_FLOATS + (has_u ? 4 * BYv * BX : 0) + (has_a ? 4 * BYv * BX : 0)) * 4u;
    int issued = 0;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int s = it % NSTv;
        const uint32_t ph = (uint32_t)(it / NSTv) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, wait_lim)) {
            *s_err = 1;
            break;
        }
        const int pid = find_problem(tbase, nprob, tile);
        const ProblemDev* P = probs + pid;
        const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P->tmaps) + mapset * NMAP;
        const int tiles_x = (P->nx + BX - 1) / BX;
        const int lt = tile - __ldg(tbase + pid);
        const int x0 = (lt % tiles_x) * BX, y0 = (lt / tiles_x) * BYv;
        fill_tile_info(info[s], P, a, x0, y0);
        float* st = smem + (size_t)s * L::FLOATS;
        mbar_expect_tx(&full[s], bytes);
        const int kx = a.x, cx = a.x == 0 ? 0 : a.x - 1;
        tma_load_4d(st + L::ZV_OFF, map_of(maps, kx, 0), x0 - TX, y0 - R, 1, cx, &full[s]);   // y_v, 2D halo
        tma_load_2d(st + L::C2_OFF, maps + 11, x0 - TX, y0 - R, &full[s]);                   // c^2, 2D halo
        tma_load_4d(st + L::WX_OFF, map_of(maps, kx, 1), x0 - TX, y0, 2, cx, &full[s]);
        tma_load_4d(st + L::WY_OFF, map_of(maps, kx, 2), x0, y0 - R, 3, cx, &full[s]);
        tma_load_4d(st + L::YU_OFF, map_of(maps, kx, 3), x0, y0, 0, cx, &full[s]);           // y_u
        if (has_u)
            tma_load_4d(st + L::PU_OFF, map_of(maps, a.u, 4), x0, y0, 0, a.u == 0 ? 0 : a.u - 1, &full[s]);
        if (has_a)
            tma_load_4d(st + L::PA_OFF, map_of(maps, a.a, 4), x0, y0, 0, a.a == 0 ? 0 : a.a - 1, &full[s]);
        issued = it + 1;
    }
    return issued;
}

// The general epilogue (StageArgs) of one point: K = cx X + ch xs HX, Y = cu U + ck K,
// ACC = ca A + cau U + cak K + cay Y + cax X, pads of w_x / w_y zero.
__device__ __forceinline__ void tma_epilogue_point(const TileInfo& ti, const StageArgs& a, long long o, const float* xf,
                                                   const float* hf, const float* uv, const float* av, bool padx,
                                                   bool pady) {
    const float chx = a.fch * ti.xs;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool pad = (f == 2 && padx) || (f == 3 && pady);
        const float kf = fmaf(a.fcx, xf[f], chx * hf[f]);
        const float yf = pad ? 0.f : (a.fcu * uv[f] + a.fck * kf);
        if (ti.Y) ti.Y[f * ti.fstr + o] = yf;
        if (ti.A)
            ti.A[f * ti.fstr + o] =
                pad ? 0.f : (a.fca * av[f] + a.fcau * uv[f] + a.fcak * kf + a.fcay * yf + a.fcax * xf[f]);
    }
}

// One transposed point from shared memory with the free-surface columns (rows 0..8 of the
// top tile), following the row structure of the forward operator.
template <int R, int BYv, bool HASU, bool HASA>
__device__ __forceinline__ void tma_point_scalar_t(const float* st, const TileInfo& ti, const StageArgs& a, int tc,
                                                   int lr, bool has_u, bool has_a) {
    using L = TLayout<R, BYv, HASU, HASA>;
    const int nx = ti.nx, ny = ti.ny;
    const int i = ti.x0 + tc, j = ti.y0 + lr;
    if (i >= nx || j >= ny) return;
    const bool fs = ti.fs != 0;
    const int cs = tc + TX;
    const float* btab = ti.btab;
    const int nbt = ti.nbtab;
    const float* zv_ = st + L::ZV_OFF;
    const float* c2_ = st + L::C2_OFF;
    const float* wx_ = st + L::WX_OFF;
    const float* wy_ = st + L::WY_OFF;
    // z_v at staged row q (grid row y0 + q - R), tile column tc + d
    auto zv = [&](int q, int d) { return zv_[q * L::SW + cs + d] * c2_[q * L::SW + cs + d]; };
    const float byn = btab_at(btab, nbt, 2 * (fs ? ny - j : min(j + 1, ny - j)));
    const float bxn = btab_at(btab, nbt, 2 * min(i + 1, nx - i));
    const float bxh = btab_at(btab, nbt, min(2 * i + 3, 2 * (nx - i) - 1));
    const float byh = btab_at(btab, nbt, fs ? 2 * (ny - j) - 1 : min(2 * j + 3, 2 * (ny - j) - 1));
    // z_x at half column i + d + 1/2 of this row, z_y at half row h of this column
    auto zx = [&](int d) {
        const int p = i + d;
        const float bh = btab_at(btab, nbt, min(2 * p + 3, 2 * (nx - p) - 1));
        return (byn - bh) * wx_[lr * L::SW + cs + d];
    };
    auto zy = [&](int h) {
        const float bh = btab_at(btab, nbt, fs ? 2 * (ny - h) - 1 : min(2 * h + 3, 2 * (ny - h) - 1));
        return (bxn - bh) * wy_[(h - ti.y0 + R) * BX + tc];
    };
    const int q0 = lr + R;   // staged row of j
    float lxx = cent<R>(0) * zv(q0, 0);
#pragma unroll
    for (int k = 1; k <= R; ++k) lxx += cent<R>(k) * (zv(q0, k) + zv(q0, -k));
    float lyy = 0.f;
    const int rfs = fs ? 4 : 0;
#pragma unroll
    for (int k = -R; k <= R; ++k) {
        const int r = j + k;
        if (r >= rfs && r < ny) lyy += cent<R>(k < 0 ? -k : k) * zv(q0 + k, 0);
    }
    if (fs && j <= 8) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < ny) lyy += g_tma_fs[TFS_UYY + r * 9 + j] * zv(r - ti.y0 + R, 0);
    }
    float gxt = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) gxt += stag<R>(k) * (zx(-1 - k) - zx(k));
    float gyt = 0.f;
    const int hfs = fs ? 3 : 0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int h1 = j + k, h2 = j - 1 - k;
        if (h1 >= hfs && h1 < ny - 1) gyt += stag<R>(k) * zy(h1);
        if (h2 >= hfs && h2 >= 0) gyt -= stag<R>(k) * zy(h2);
    }
    if (fs && j <= 7) {
#pragma unroll
        for (int h = 0; h < 3; ++h)
            if (h < ny - 1) gyt += g_tma_fs[TFS_UY + h * 8 + j] * zy(h);
    }
    float dxt = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) dxt += stag<R>(k) * (zv(q0, -k) - zv(q0, 1 + k));
    float dyt = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r1 = j + 1 + k, r2 = j - k;
        if (r1 >= rfs && r1 < ny) dyt += stag<R>(k) * zv(q0 + 1 + k, 0);
        if (r2 >= rfs && r2 >= 0) dyt -= stag<R>(k) * zv(q0 - k, 0);
    }
    if (fs && j <= 7) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < ny) dyt += g_tma_fs[TFS_DWY + r * 8 + j] * zv(r - ti.y0 + R, 0);
    }
    const int pt = lr * BX + tc;
    const float yu = st[L::YU_OFF + pt], yv = zv_[q0 * L::SW + cs];
    const float ywx = (i < nx - 1) ? wx_[lr * L::SW + cs] : 0.f;
    const float ywy = (j < ny - 1) ? wy_[q0 * BX + tc] : 0.f;
    const float idx1 = ti.idx1, idx2 = ti.idx2;
    const float xf[4] = {yu, yv, ywx, ywy};
    const float hf[4] = {-bxn * byn * yv + (lxx + lyy) * idx2 + (gxt + gyt) * idx1, yu - (bxn + byn) * yv,
                         (i < nx - 1) ? dxt * idx1 - bxh * ywx : 0.f, (j < ny - 1) ? dyt * idx1 - byh * ywy : 0.f};
    float uv[4], av[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        uv[f] = has_u ? st[L::PU_OFF + f * BYv * BX + pt] : 0.f;
        av[f] = has_a ? st[L::PA_OFF + f * BYv * BX + pt] : 0.f;
    }
    tma_epilogue_point(ti, a, (long long)j * ti.pitch + i, xf, hf, uv, av, i >= nx - 1, j >= ny - 1);
}

template <int R, int BYv, int NW, int NSTv, bool HASU, bool HASA>
__global__ void __launch_bounds__(NW * 32 + 32, 1)
stage_tma_t_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tbase, int nprob, int ntiles,
                   int mapset, StageArgs a, int* err) {
    using L = TLayout<R, BYv, HASU, HASA>;
    constexpr int CPR = BX / 2;
    constexpr int TPR = NW * 32 / CPR;
    constexpr int NR = BYv / TPR;
    static_assert(NR * TPR == BYv && NR >= 1, "tile rows must split evenly over threads");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NSTv];
    __shared__ __align__(8) uint64_t empty[NSTv];
    __shared__ TileInfo info[NSTv];
    __shared__ int s_err;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint64_t wait_lim = g_tma_wait_limit_ns;
    if (tid == 0) {
        for (int s = 0; s < NSTv; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool has_u = HASU && a.u >= 0, has_a = HASA && a.a >= 0;
    int issued = 0;
    if (warp == NW) {
        if (lane == 0)
            issued = tma_produce_t<R, BYv, NSTv, HASU, HASA>(probs, tbase, nprob, ntiles, mapset, a, smem, full,
                                                             empty, info, &s_err, wait_lim);
    } else {
        const int tx2 = tid % CPR, ty = tid / CPR;
        const int c0 = 2 * tx2, cs = c0 + TX, r0 = NR * ty;
        const float2 cx2 = f2s(a.fcx), cu2 = f2s(a.fcu), ck2 = f2s(a.fck), ca2 = f2s(a.fca);
        const float2 cay2 = f2s(a.fcay), cau2 = f2s(a.fcau), cak2 = f2s(a.fcak), cax2 = f2s(a.fcax);
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it % NSTv;
            const uint32_t ph = (uint32_t)(it / NSTv) & 1u;
            if (!mbar_wait(&full[s], ph, wait_lim)) {
                s_err = 1;
                break;
            }
            const TileInfo ti = load_info(&info[s]);
            const float* st = smem + (size_t)s * L::FLOATS;
            const int nx = ti.nx, ny = ti.ny;
            const int i0 = ti.x0 + c0;
            const int jt = ti.y0 + r0;
            if (i0 < nx && jt < ny) {
                if (ti.fs != 0 && jt < 9) {
#pragma unroll 1
                    for (int r = 0; r < NR; ++r) {
                        tma_point_scalar_t<R, BYv, HASU, HASA>(st, ti, a, c0, r0 + r, has_u, has_a);
                        tma_point_scalar_t<R, BYv, HASU, HASA>(st, ti, a, c0 + 1, r0 + r, has_u, has_a);
                    }
                } else {
                    const float* zvp = st + L::ZV_OFF;
                    const float* c2p = st + L::C2_OFF;
                    const float* wxp = st + L::WX_OFF;
                    const float* wyp = st + L::WY_OFF;
                    const float* yup = st + L::YU_OFF;
                    const float* spu = st + L::PU_OFF;
                    const float* spa = st + L::PA_OFF;
                    const bool fs = ti.fs != 0;
                    const bool in1 = i0 + 1 < nx;
                    const float* btab = ti.btab;
                    const int nbt = ti.nbtab;
                    const float2 bxn = f2(btab_at(btab, nbt, 2 * min(i0 + 1, nx - i0)),
                                          btab_at(btab, nbt, 2 * min(i0 + 2, nx - i0 - 1)));
                    // bx at the half columns i0 + d + 1/2, d = -4 .. 5 (the z_x taps)
                    float bxh[10];
#pragma unroll
                    for (int d = -4; d <= 5; ++d) {
                        const int p = i0 + d;
                        bxh[d + 4] = btab_at(btab, nbt, min(2 * p + 3, 2 * (nx - p) - 1));
                    }
                    const float2 bxhp = f2(bxh[4], bxh[5]);   // at this thread's two columns
                    unsigned xin = 0u;                           // half columns 0 .. nx - 2
#pragma unroll
                    for (int d = -4; d <= 5; ++d)
                        if (i0 + d >= 0 && i0 + d < nx - 1) xin |= 1u << (d + 4);
                    // z_v = c^2 y_v and z_y = (bx - by^h) y_wy down this column pair
                    float2 zq[NR + 2 * R], zyq[NR + 2 * R - 1];
#pragma unroll
                    for (int q = 0; q < NR + 2 * R; ++q)
                        zq[q] = mul2(lds2(zvp + (r0 + q) * L::SW + cs), lds2(c2p + (r0 + q) * L::SW + cs));
#pragma unroll
                    for (int q = 0; q < NR + 2 * R - 1; ++q) {
                        const int h = ti.y0 + r0 + q - R;
                        const float bh = btab_at(btab, nbt, fs ? 2 * (ny - h) - 1 : min(2 * h + 3, 2 * (ny - h) - 1));
                        zyq[q] = (h >= 0 && h < ny - 1) ? mul2(sub2(bxn, f2s(bh)), lds2(wyp + (r0 + q) * BX + c0))
                                                        : f2s(0.f);
                    }
                    const bool wx0in = i0 < nx - 1, wx1in = i0 + 1 < nx - 1;
                    const float2 idx1 = f2s(ti.idx1), idx2 = f2s(ti.idx2);
                    const float2 chx2 = f2s(a.fch * ti.xs);
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int lr = r0 + r, j = jt + r;
                        if (j >= ny) break;
                        const float byn = btab_at(btab, nbt, 2 * (fs ? ny - j : min(j + 1, ny - j)));
                        const float byh =
                            btab_at(btab, nbt, fs ? 2 * (ny - j) - 1 : min(2 * j + 3, 2 * (ny - j) - 1));
                        // x taps of z_v (pairs at column offsets -4 .. 5) and y_wx
                        const float* zr = zvp + (lr + R) * L::SW + cs;
                        const float* cr = c2p + (lr + R) * L::SW + cs;
                        const float2 zp[5] = {mul2(lds2(zr - 4), lds2(cr - 4)), mul2(lds2(zr - 2), lds2(cr - 2)),
                                              zq[r + R], mul2(lds2(zr + 2), lds2(cr + 2)),
                                              mul2(lds2(zr + 4), lds2(cr + 4))};
                        const float* wr = wxp + lr * L::SW + cs;
                        const float2 wp[5] = {lds2(wr - 4), lds2(wr - 2), lds2(wr), lds2(wr + 2), lds2(wr + 4)};
                        auto zo = [&](int d) { return ((d + 4) & 1) ? zp[(d + 4) >> 1].y : zp[(d + 4) >> 1].x; };
                        // z_x at half column offset d: (by - bx^h) y_wx (zero off the w_x grid)
                        auto xo = [&](int d) {
                            const float wv = ((d + 4) & 1) ? wp[(d + 4) >> 1].y : wp[(d + 4) >> 1].x;
                            return ((xin >> (d + 4)) & 1u) ? (byn - bxh[d + 4]) * wv : 0.f;
                        };
                        const float2 zc = zq[r + R];
                        float2 lap = mul2(f2s(2.f * cent<R>(0)), zc);
                        float2 gxt = f2s(0.f), gyt = f2s(0.f), dxt = f2s(0.f), dyt = f2s(0.f);
#pragma unroll
                        for (int k = 0; k < R; ++k) {
                            const int kk = k + 1;
                            const float2 sx = (kk & 1) ? f2(zo(kk) + zo(-kk), zo(kk + 1) + zo(1 - kk))
                                                       : add2(zp[(kk + 4) >> 1], zp[(4 - kk) >> 1]);
                            const float2 sy = add2(zq[r + R + kk], zq[r + R - kk]);
                            lap = fma2(f2s(cent<R>(kk)), add2(sx, sy), lap);
                            gxt = fma2(f2s(stag<R>(k)), f2(xo(-1 - k) - xo(k), xo(-k) - xo(1 + k)), gxt);
                            gyt = fma2(f2s(stag<R>(k)), sub2(zyq[r + R + k], zyq[r + R - 1 - k]), gyt);
                            dxt = fma2(f2s(stag<R>(k)), f2(zo(-k) - zo(1 + k), zo(1 - k) - zo(2 + k)), dxt);
                            dyt = fma2(f2s(stag<R>(k)), sub2(zq[r + R + 1 + k], zq[r + R - k]), dyt);
                        }
                        const int pt = lr * BX + c0;
                        const float2 yv = lds2(zvp + (lr + R) * L::SW + cs);
                        const float2 yu = lds2(yup + pt);
                        const bool wyin = j < ny - 1;
                        float2 ywx = wp[2];
                        if (!wx0in) ywx.x = 0.f;
                        if (!wx1in) ywx.y = 0.f;
                        const float2 ywy = wyin ? lds2(wyp + (lr + R) * BX + c0) : f2s(0.f);
                        // (H^T y)_u, _v, _wx, _wy
                        const float2 hu = fma2(mul2(bxn, f2s(-byn)), yv,
                                               fma2(lap, idx2, mul2(add2(gxt, gyt), idx1)));
                        const float2 hv = fma2(sub2(f2s(-byn), bxn), yv, yu);
                        float2 hwx = fma2(dxt, idx1, mul2(f2(-bxhp.x, -bxhp.y), ywx));
                        if (!wx0in) hwx.x = 0.f;
                        if (!wx1in) hwx.y = 0.f;
                        const float2 hwy = wyin ? fma2(dyt, idx1, mul2(f2s(-byh), ywy)) : f2s(0.f);
                        const float2 xf[4] = {yu, yv, ywx, ywy};
                        const float2 hf[4] = {hu, hv, hwx, hwy};
                        const long long o = (long long)j * ti.pitch + i0;
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            const float2 uval = has_u ? lds2(spu + f * BYv * BX + pt) : f2s(0.f);
                            const float2 aval = has_a ? lds2(spa + f * BYv * BX + pt) : f2s(0.f);
                            const float2 kf = fma2(cx2, xf[f], mul2(chx2, hf[f]));
                            float2 yf = fma2(cu2, uval, mul2(ck2, kf));
                            float2 af = fma2(cax2, xf[f],
                                             fma2(cay2, yf, fma2(cak2, kf, fma2(cau2, uval, mul2(ca2, aval)))));
                            if (f == 2) {
                                if (!wx0in) yf.x = af.x = 0.f;
                                if (!wx1in) yf.y = af.y = 0.f;
                            }
                            if (f == 3 && !wyin) yf = af = f2s(0.f);
                            if (ti.Y) st2(ti.Y + f * ti.fstr + o, yf, in1);
                            if (ti.A) st2(ti.A + f * ti.fstr + o, af, in1);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    tma_finish<NSTv>(s_err, issued, full, err);
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encoder() {
    if (g_encode) return 0;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return -1;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return 0;
}

// 4D map over (x, y, field, vector) of one buffer, box (bx, by, bf, 1).
static int encode4(CUtensorMap* out, void* base, int nx, int ny, int nvec, long long pitch,
                   long long fstride, long long vstride, int bx, int by, int bf) {
    cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, 4, (cuuint64_t)nvec};
    cuuint64_t strides[3] = {(cuuint64_t)pitch * 4, (cuuint64_t)fstride * 4, (cuuint64_t)vstride * 4};
    cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bf, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

static int encode2(CUtensorMap* out, void* base, int nx, int ny, long long pitch, int bx, int by) {
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int tma_map_set(int tile_height) {
    for (int k = 0; k < TMA_NUM_SETS; ++k)
        if (TMA_SET_HEIGHTS[k] == tile_height) return k;
    return -1;
}
constexpr int map_set_of(int by) {
    for (int k = 0; k < TMA_NUM_SETS; ++k)
        if (TMA_SET_HEIGHTS[k] == by) return k;
    return -1;
}
static_assert(map_set_of(16) == 0 && map_set_of(18) == 3 && map_set_of(24) >= 0 && map_set_of(28) >= 0 &&
                  map_set_of(30) >= 0 && map_set_of(36) >= 0,
              "every tile height in use has a map set");

// Build NMAP maps per problem and tile height (one map set per entry of TMA_SET_HEIGHTS)
// into a device array (FP32 only); sets P.tmaps to the problem's first map.
int build_tensor_maps(std::vector<ProblemDev>& probs, int R, const std::vector<int>& work_vecs,
                      void** d_maps_inout) {
    if (get_encoder() != 0) return -1;
    const int n = (int)probs.size();
    constexpr int NSET = TMA_NUM_SETS;
    const int* heights = TMA_SET_HEIGHTS;
    std::vector<CUtensorMap> maps((size_t)n * NSET * NMAP);
    const int SW = BX + 2 * TX;
    for (int p = 0; p < n; ++p) {
        ProblemDev& P = probs[p];
        for (int set = 0; set < NSET; ++set) {
            const int by = heights[set], SH = by + 2 * R;
            CUtensorMap* m = maps.data() + ((size_t)p * NSET + set) * NMAP;
            const int bxs[5] = {SW, SW, BX, BX, BX};
            const int bys[5] = {SH, by, SH, by, by};
            const int bfs[5] = {1, 1, 1, 1, 4};
            for (int k = 0; k < 5; ++k) {
                if (encode4(m + k, P.state, P.nx, P.ny, 1, P.pitch, P.field_stride, P.vec_stride,
                            bxs[k], bys[k], bfs[k]) != 0)
                    return -1;
                void* wb = P.work ? P.work : P.state;
                const int nv = P.work ? work_vecs[p] : 1;
                if (encode4(m + 5 + k, wb, P.nx, P.ny, nv > 0 ? nv : 1, P.pitch, P.field_stride,
                            P.vec_stride, bxs[k], bys[k], bfs[k]) != 0)
                    return -1;
            }
            if (encode2(m + 10, const_cast<void*>(P.c2), P.nx, P.ny, P.pitch, BX, by) != 0) return -1;
            // c^2 with the 2D halo of u (the transposed pass stages c^2 y_v)
            if (encode2(m + 11, const_cast<void*>(P.c2), P.nx, P.ny, P.pitch, SW, SH) != 0) return -1;
        }
    }
    cudaFree(*d_maps_inout);
    *d_maps_inout = nullptr;
    if (cudaMalloc(d_maps_inout, sizeof(CUtensorMap) * maps.size()) != cudaSuccess) return -1;
    if (cudaMemcpy(*d_maps_inout, maps.data(), sizeof(CUtensorMap) * maps.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return -1;
    for (int p = 0; p < n; ++p)
        probs[p].tmaps = static_cast<char*>(*d_maps_inout) + (size_t)p * NSET * NMAP * sizeof(CUtensorMap);
    return 0;
}

// Kernel variants the autotuner chooses from: (tile height, consumer warps, stages).  Variant
// 4 has no U buffer (4 stages of 64 x 16): passes with a U operand run variant 0 instead.
// Variant 5 keeps two rows per consumer thread with 20 warps (64 x 20 tiles): 21 warps per
// SM, which caps a thread at 80 registers (six warps share one scheduler's register file).
// Variant 6 uses 18 warps (64 x 18 tiles): 19 warps per SM, still 96 registers a thread.
// Variants 7 to 9 run the column-pair consumers (two columns per thread): 7 = 64 x 18 tiles
// with 9 warps (two rows a thread), 8 = 64 x 16 with 8 warps (two rows), 9 = 64 x 18 with
// 18 warps (one row), 10 = 64 x 24 with 12 warps and 2 stages (two rows).  11 and 12 are
// composite: passes that read an A operand run variant 7, the others (Horner HORK passes,
// Krylov products, leap-frog-free RK stages without an accumulator) drop the A buffer and
// take taller tiles: 11 = 64 x 24 with 12 warps and 3 stages, 12 = 64 x 36 with 9 warps, four
// rows a thread and 2 stages; 13 = 64 x 28 with 14 warps and 3 stages; 14 = 64 x 30 with 15
// warps and 3 stages (512 threads at 128 registers: the whole register file).  The shape
// reported for a composite is its no-A shape.
struct TmaVariant {
    int by, nw, nst;
};
constexpr TmaVariant kVariants[TMA_NUM_VARIANTS] = {
    {16, 16, 3}, {16, 8, 3}, {8, 8, 5},  {8, 16, 5},  {16, 16, 4}, {20, 20, 3}, {18, 18, 3},
    {18, 9, 3},  {16, 8, 3}, {18, 18, 3}, {24, 12, 2}, {24, 12, 3}, {36, 9, 2}, {28, 14, 3}, {30, 15, 3}};

static bool composite(int v) { return v >= 11 && v <= 14; }

int tma_variant_tile_height_for(int v, bool reads_a) {
    if (composite(v) && reads_a) return kVariants[7].by;
    return kVariants[v].by;
}

int tma_variant_tile_height(int v) { return kVariants[v].by; }
void tma_variant_describe(int v, int* by, int* nw, int* nst) {
    *by = kVariants[v].by;
    *nw = kVariants[v].nw;
    *nst = kVariants[v].nst;
}

static int g_num_sms = 0;

template <int R, int BYv, int NW, int NSTv, int EPI, bool HASU = true>
static int launch_variant(const ProblemDev* probs, const int* tbase, int nprob, int ntiles,
                          const StageArgs& a, int* err, cudaStream_t s) {
    const size_t smem = (size_t)NSTv * StageLayout<R, BYv, HASU>::BYTES + 1024;
    // the shared-memory attribute is set once per instantiation and device
    static unsigned long long configured = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    if (!(configured >> dev & 1ull)) {
        if (cudaFuncSetAttribute(stage_tma_kernel<R, BYv, NW, NSTv, EPI, HASU>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
        configured |= 1ull << dev;
    }
    const int grid = ntiles < g_num_sms ? ntiles : g_num_sms;
    stage_tma_kernel<R, BYv, NW, NSTv, EPI, HASU><<<grid, NW * 32 + 32, smem, s>>>(
        probs, tbase, nprob, ntiles, map_set_of(BYv), a, err);
    return 0;
}

template <int R, int BYv, int NW, int NSTv, int EPI, bool HASA = true, bool HASU = true>
static int launch_x2(const ProblemDev* probs, const int* tbase, int nprob, int ntiles, const StageArgs& a,
                     int* err, cudaStream_t s) {
    static_assert(map_set_of(BYv) >= 0, "tile height without a map set");
    if (!HASA && a.a >= 0) return -1;    // a pass with an A operand needs the A buffer
    if (!HASU && a.u >= 0) return -1;    // and one with a U operand the U buffer
    const size_t smem = (size_t)NSTv * StageLayout<R, BYv, HASU, HASA>::BYTES + 1024;
    static unsigned long long configured = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    if (!(configured >> dev & 1ull)) {
        if (cudaFuncSetAttribute(stage_tma_x2_kernel<R, BYv, NW, NSTv, EPI, HASU, HASA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
        configured |= 1ull << dev;
    }
    const int grid = ntiles < g_num_sms ? ntiles : g_num_sms;
    stage_tma_x2_kernel<R, BYv, NW, NSTv, EPI, HASU, HASA><<<grid, NW * 32 + 32, smem, s>>>(
        probs, tbase, nprob, ntiles, map_set_of(BYv), a, err);
    return 0;
}

// One leap-frog step (EPI 2) on the column-pair consumers (64 x 30 tiles, 15 warps, 3
// stages, no U buffer); tbase and ntiles are those of the 30-row map set.
int launch_leapfrog_tma(int R, const ProblemDev* probs, const int* tbase, int nprob, int ntiles, int cur,
                        int prev, int variant, double dt, int* err, cudaStream_t s) {
    if (ntiles <= 0) return nprob > 0 ? -1 : 0;
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    StageArgs a{};
    a.x = cur;
    a.u = -1;
    a.a = prev;
    a.y_out = prev;
    a.acc_out = cur;
    a.d = -1;
    a.src_slot = 0;
    a.x_scale_slot = -1;
    a.m = variant;
    a.dt = dt;
    if (R == 4) return launch_x2<4, 30, 15, 3, 2, true, false>(probs, tbase, nprob, ntiles, a, err, s);
    if (R == 2) return launch_x2<2, 30, 15, 3, 2, true, false>(probs, tbase, nprob, ntiles, a, err, s);
    return -1;
}

// The FWI gradient pass (EPI 3): grad += gscale q_v (L u + D w) of vector a.x, q = a.gq (its
// four fields ride in the A box); column-pair consumers on the leap-frog step's tiles
// (64 x 30, 15 warps, 3 stages; the 30-row map set).
int launch_grad_tma(int R, const ProblemDev* probs, const int* tbase, int nprob, int ntiles,
                    const StageArgs& a_in, int* err, cudaStream_t s) {
    if (ntiles <= 0) return nprob > 0 ? -1 : 0;
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    StageArgs a = a_in;
    a.u = -1;
    a.a = a.gq;
    a.y_out = -1;
    a.acc_out = -1;
    if (R == 4) return launch_x2<4, 30, 15, 3, 3, true, false>(probs, tbase, nprob, ntiles, a, err, s);
    if (R == 2) return launch_x2<2, 30, 15, 3, 3, true, false>(probs, tbase, nprob, ntiles, a, err, s);
    return -1;
}

template <int R, bool HASU, bool HASA>
static int launch_t(const ProblemDev* probs, const int* tbase, int nprob, int ntiles, const StageArgs& a, int* err,
                    cudaStream_t s) {
    constexpr int BYv = 18, NW = 9, NSTv = 3;
    const size_t smem = (size_t)NSTv * TLayout<R, BYv, HASU, HASA>::BYTES + 1024;
    static unsigned long long configured = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    if (!(configured >> dev & 1ull)) {
        if (cudaFuncSetAttribute(stage_tma_t_kernel<R, BYv, NW, NSTv, HASU, HASA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
        configured |= 1ull << dev;
    }
    const int grid = ntiles < g_num_sms ? ntiles : g_num_sms;
    stage_tma_t_kernel<R, BYv, NW, NSTv, HASU, HASA><<<grid, NW * 32 + 32, smem, s>>>(
        probs, tbase, nprob, ntiles, map_set_of(BYv), a, err);
    return 0;
}

// The transposed pass H^T (FP32, no dot partner, no gradient) on 64 x 18 tiles with 9
// column-pair consumer warps; tbase and ntiles are those of the 18-row map set.
int launch_transpose_tma(int R, const ProblemDev* probs, const int* tbase, int nprob, int ntiles,
                         const StageArgs& a_in, int* err, cudaStream_t s) {
    if (ntiles <= 0) return nprob > 0 ? -1 : 0;
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    StageArgs a = a_in;
    a.fcx = (float)a.cx;
    a.fch = (float)a.ch;
    a.fcu = (float)a.cu;
    a.fck = (float)a.ck;
    a.fca = (float)a.ca;
    a.fcau = (float)a.cau;
    a.fcak = (float)a.cak;
    a.fcay = (float)a.cay;
    a.fcax = (float)a.cax;
    const bool hu = a.u >= 0, ha = a.a >= 0;
    if (R == 4)
        return hu ? (ha ? launch_t<4, true, true>(probs, tbase, nprob, ntiles, a, err, s)
                        : launch_t<4, true, false>(probs, tbase, nprob, ntiles, a, err, s))
                  : (ha ? launch_t<4, false, true>(probs, tbase, nprob, ntiles, a, err, s)
                        : launch_t<4, false, false>(probs, tbase, nprob, ntiles, a, err, s));
    if (R == 2)
        return hu ? (ha ? launch_t<2, true, true>(probs, tbase, nprob, ntiles, a, err, s)
                        : launch_t<2, true, false>(probs, tbase, nprob, ntiles, a, err, s))
                  : (ha ? launch_t<2, false, true>(probs, tbase, nprob, ntiles, a, err, s)
                        : launch_t<2, false, false>(probs, tbase, nprob, ntiles, a, err, s));
    return -1;
}

int launch_stage_tma(int variant, int R, const ProblemDev* probs, const int* tbase, int nprob,
                     int ntiles, const StageArgs& a_in, int* err, cudaStream_t s) {
    StageArgs a = a_in;
    a.fcx = (float)a.cx;
    a.fch = (float)a.ch;
    a.fcu = (float)a.cu;
    a.fck = (float)a.ck;
    a.fca = (float)a.ca;
    a.fcau = (float)a.cau;
    a.fcak = (float)a.cak;
    a.fcay = (float)a.cay;
    a.fcax = (float)a.cax;
    if (ntiles <= 0) return nprob > 0 ? -1 : 0;   // problems but no tiles: inconsistent lists
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    // the steady-state Faber / HORK form: Y = cu U + cx X + ch H, ACC = ca A + cay Y
    const bool epi = a.ck == 1.0 && a.cau == 0.0 && a.cak == 0.0 && a.cax == 0.0;
#define EWV_TMA_CASE(V, RR, BYV, NWV, NSTV) \
    if (variant == V && R == RR)                                                                \
        return epi ? launch_variant<RR, BYV, NWV, NSTV, 1>(probs, tbase, nprob, ntiles, a, err, s) \
                   : launch_variant<RR, BYV, NWV, NSTV, 0>(probs, tbase, nprob, ntiles, a, err, s);
    EWV_TMA_CASE(0, 4, 16, 16, 3)
    EWV_TMA_CASE(1, 4, 16, 8, 3)
    EWV_TMA_CASE(2, 4, 8, 8, 5)
    EWV_TMA_CASE(3, 4, 8, 16, 5)
    EWV_TMA_CASE(5, 4, 20, 20, 3)
    EWV_TMA_CASE(6, 4, 18, 18, 3)
#define EWV_TMA_X2_CASE(V, RR, BYV, NWV, NSTV) \
    if (variant == V && R == RR)                                                             \
        return epi ? launch_x2<RR, BYV, NWV, NSTV, 1>(probs, tbase, nprob, ntiles, a, err, s) \
                   : launch_x2<RR, BYV, NWV, NSTV, 0>(probs, tbase, nprob, ntiles, a, err, s);
    if (composite(variant) && a.a >= 0) variant = 7;   // composite, pass with A
#define EWV_TMA_X2_NOA_CASE(V, RR, BYV, NWV, NSTV) \
    if (variant == V && R == RR)                                                                    \
        return epi ? launch_x2<RR, BYV, NWV, NSTV, 1, false>(probs, tbase, nprob, ntiles, a, err, s) \
                   : launch_x2<RR, BYV, NWV, NSTV, 0, false>(probs, tbase, nprob, ntiles, a, err, s);
    EWV_TMA_X2_CASE(7, 4, 18, 9, 3)
    EWV_TMA_X2_CASE(8, 4, 16, 8, 3)
    EWV_TMA_X2_CASE(9, 4, 18, 18, 3)
    EWV_TMA_X2_CASE(10, 4, 24, 12, 2)
    EWV_TMA_X2_NOA_CASE(11, 4, 24, 12, 3)
    EWV_TMA_X2_NOA_CASE(12, 4, 36, 9, 2)
    EWV_TMA_X2_NOA_CASE(13, 4, 28, 14, 3)
    EWV_TMA_X2_NOA_CASE(14, 4, 30, 15, 3)
    EWV_TMA_X2_CASE(7, 2, 18, 9, 3)
    EWV_TMA_X2_CASE(8, 2, 16, 8, 3)
    EWV_TMA_X2_CASE(9, 2, 18, 18, 3)
    EWV_TMA_X2_CASE(10, 2, 24, 12, 2)
    EWV_TMA_X2_NOA_CASE(11, 2, 24, 12, 3)
    EWV_TMA_X2_NOA_CASE(12, 2, 36, 9, 2)
    EWV_TMA_X2_NOA_CASE(13, 2, 28, 14, 3)
    EWV_TMA_X2_NOA_CASE(14, 2, 30, 15, 3)
#undef EWV_TMA_X2_NOA_CASE
#undef EWV_TMA_X2_CASE
    if (variant == 4) {   // no U buffer; a pass with a U operand runs variant 0
        if (a.u >= 0) variant = 0;
        else if (R == 4)
            return epi ? launch_variant<4, 16, 16, 4, 1, false>(probs, tbase, nprob, ntiles, a, err, s)
                       : launch_variant<4, 16, 16, 4, 0, false>(probs, tbase, nprob, ntiles, a, err, s);
        else
            return epi ? launch_variant<2, 16, 16, 4, 1, false>(probs, tbase, nprob, ntiles, a, err, s)
                       : launch_variant<2, 16, 16, 4, 0, false>(probs, tbase, nprob, ntiles, a, err, s);
    }
    EWV_TMA_CASE(0, 4, 16, 16, 3)
    EWV_TMA_CASE(0, 2, 16, 16, 3)
    EWV_TMA_CASE(1, 2, 16, 8, 3)
    EWV_TMA_CASE(2, 2, 8, 8, 5)
    EWV_TMA_CASE(3, 2, 8, 16, 5)
    EWV_TMA_CASE(5, 2, 20, 20, 3)
    EWV_TMA_CASE(6, 2, 18, 18, 3)
#undef EWV_TMA_CASE
    return -1;
}

}  // namespace ewv
