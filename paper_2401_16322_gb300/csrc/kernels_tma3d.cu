// Persistent, TMA-fed fused stencil pass for three-dimensional problems (FP32, forward
// operator) on sm_103a.
//
// Same arithmetic as stage3d_kernel (kernels_3d.cu: the three-dimensional PML form of Eq. 1
// with the auxiliary field psi, Sec. 2.1 stencils, Appendix A / Sec. 2.2 rows on the vertical
// axis, damping from the per-model table, and the integrators' K / Y / ACC epilogue),
// organised for HBM bandwidth:
//   - a task is one 64 x 8 column tile of one problem over a chunk of KC3 planes; one CTA per
//     SM walks the task list (tasks b, b + gridDim.x, ...);
//   - the producer lane streams the chunk plane by plane through NST shared-memory stages
//     (cp.async.bulk.tensor over 5D maps: x, y, z, field, vector).  The stage for compute
//     plane c holds u(c) with its x / y halo, w_x(c) (x halo), w_y(c) (y halo), v(c), c^2(c),
//     psi(c), the six-field pointwise operands U(c) and A(c), and the "front" values
//     u(c + R) and w_z(c + R - 1);
//   - the psi derivatives are needed only where a product of two damping coefficients is
//     nonzero (the edges of the layer): there they are read with plain loads;
//   - 2R warm-up stages before a chunk's first plane carry only front values;
//   - the consumer warps push the front values into per-thread register queues
//     (u over c-R .. c+R, w_z over c-R .. c+R-1), which supply every vertical tap.  The
//     x and y taps come from the staged plane.  Y / ACC are stored with coalesced st.global.
// TMA zero fill outside the tensor is the zero extension; the w_z pad plane (k = nz-1) holds
// zeros.  The free-surface rows (planes 0..3) read their column taps with plain loads.
// Every mbarrier wait is bounded (1 s of %globaltimer); on expiry the kernel records an
// error word, drains its own copies (bounded) and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <vector>

#include "ewave_internal.cuh"

namespace ewv {

namespace {

constexpr int TX3 = 4;      // staged x halo (>= R, keeps the box start 16-byte aligned)
constexpr int BY3 = 8;      // tile height of this kernel
constexpr int NMAP3 = 11;   // tensor maps per problem

template <int R>
struct Stage3 {
    static constexpr int SH = BY3 + 2 * R;
    static constexpr int SW = BX + 2 * TX3;
    static constexpr int PL = BY3 * BX;                  // one plane of the tile
    static constexpr int U_OFF = 0;                      // u(c)      SH x SW
    static constexpr int UF_OFF = U_OFF + SH * SW;       // u(c+R)    PL
    static constexpr int WZ_OFF = UF_OFF + PL;           // w_z(c+R-1) PL
    static constexpr int WX_OFF = WZ_OFF + PL;           // w_x(c)    BY3 x SW
    static constexpr int WY_OFF = WX_OFF + BY3 * SW;     // w_y(c)    SH x BX
    static constexpr int V_OFF = WY_OFF + SH * BX;       // v(c)      PL
    static constexpr int C2_OFF = V_OFF + PL;            // c^2(c)    PL
    static constexpr int PS_OFF = C2_OFF + PL;           // psi(c)    PL
    static constexpr int PU_OFF = PS_OFF + PL;           // U(c)      6 x PL
    static constexpr int PA_OFF = PU_OFF + 6 * PL;       // A(c)      6 x PL
    static constexpr int FLOATS = PA_OFF + 6 * PL;
    static constexpr int BYTES = FLOATS * 4;
    static_assert((UF_OFF * 4) % 128 == 0 && (WZ_OFF * 4) % 128 == 0 && (WX_OFF * 4) % 128 == 0 &&
                      (WY_OFF * 4) % 128 == 0 && (V_OFF * 4) % 128 == 0 &&
                      (C2_OFF * 4) % 128 == 0 && (PS_OFF * 4) % 128 == 0 && (PU_OFF * 4) % 128 == 0 &&
                      (PA_OFF * 4) % 128 == 0 && BYTES % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
};

struct __align__(16) Info3 {
    float* Y;
    float* A;
    const float* X;          // u field of the input vector (free-surface column taps)
    long long fstr, ps;
    int x0, y0, c, warm;     // compute plane c; warm = 1: front values only
    int nx, ny, nz, pitch, pml, fs, src_i, src_j, src_k, pad0;
    float beta0, inv_pml, idx1, idx2, sig, xs;   // xs: per-problem scale of H X (Krylov)
};

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false after 1 s (or 2^26 polls) without the phase completing.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    if (bar_try_wait(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (bar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && now_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}
__device__ __forceinline__ void tma5(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                     int c3, int c4, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                     uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
        : "memory");
}

__constant__ float g3t_fs[4 * 9 + 3 * 8 + 4 * 8];
constexpr int T3_UZZ = 0, T3_UZ = 36, T3_DWZ = 60;

template <int R>
__device__ __forceinline__ float st3(int k) {
    if constexpr (R == 4) {
        return k == 0 ? float(1225.0 / 1024.0) : k == 1 ? float(-245.0 / 3072.0)
             : k == 2 ? float(49.0 / 5120.0) : float(-5.0 / 7168.0);
    } else {
        return k == 0 ? float(9.0 / 8.0) : float(-1.0 / 24.0);
    }
}
template <int R>
__device__ __forceinline__ float ce3(int k) {
    if constexpr (R == 4) {
        return k == 0 ? float(-205.0 / 72.0) : k == 1 ? float(8.0 / 5.0) : k == 2 ? float(-1.0 / 5.0)
             : k == 3 ? float(8.0 / 315.0) : float(-1.0 / 560.0);
    } else {
        return k == 0 ? float(-5.0 / 2.0) : k == 1 ? float(4.0 / 3.0) : float(-1.0 / 12.0);
    }
}
// Stencil sums as balanced trees (short dependency chains): st_tree = sum_k s_k d[k] over the
// R staggered differences, ce_tree = c_0 u + sum_k c_k p[k-1] over the R symmetric pair sums.
template <int R>
__device__ __forceinline__ float st_tree(const float (&d)[R]) {
    if constexpr (R == 4)
        return fmaf(st3<4>(0), d[0], st3<4>(1) * d[1]) + fmaf(st3<4>(2), d[2], st3<4>(3) * d[3]);
    else
        return fmaf(st3<R>(0), d[0], st3<R>(1) * d[1]);
}
template <int R>
__device__ __forceinline__ float ce_tree(float u, const float (&p)[R]) {
    if constexpr (R == 4)
        return (fmaf(ce3<4>(1), p[0], ce3<4>(0) * u) + fmaf(ce3<4>(3), p[2], ce3<4>(2) * p[1])) +
               ce3<4>(4) * p[3];
    else
        return fmaf(ce3<R>(1), p[0], ce3<R>(0) * u) + ce3<R>(2) * p[1];
}

// beta at 2 d = k half cells from the first ghost line, from the model's table (zero beyond
// the layer; negative k, from rows and columns past a ragged grid edge, also gives zero)
__device__ __forceinline__ float bt3(const float* t, int n, int k) {
    return (unsigned)k < (unsigned)n ? __ldg(t + k) : 0.f;
}

__device__ __forceinline__ float dmp(float beta0, float inv_pml, float d, int pml) {
    if (pml <= 0) return 0.f;
    const float r = 1.f - d * inv_pml;
    return (d <= (float)pml) ? beta0 * r * r : 0.f;
}

// Half-point derivative of psi along one axis (unscaled), plain loads: p points at psi of the
// output node, `stride` is the axis stride, idx the node index and n the extent (zero
// extension); up = true for the vertical axis (sum_q s_q (psi_{k-q} - psi_{k+1+q})).
template <int R>
__device__ __forceinline__ float dpsi3(const float* p, long long stride, int idx, int n, bool up) {
    float d[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const float fwd = (idx + 1 + q < n) ? __ldg(p + (long long)(1 + q) * stride) : 0.f;
        const float bwd = (idx - q >= 0) ? __ldg(p - (long long)q * stride) : 0.f;
        d[q] = up ? bwd - fwd : fwd - bwd;
    }
    return st_tree<R>(d);
}

// Map `kind` (0 u halo box, 1 w_x box, 2 w_y box, 3 one-field plane, 4 six-field plane) of
// vector k; map 10 is c^2.
__device__ __forceinline__ const CUtensorMap* map3(const CUtensorMap* base, int k, int kind) {
    return base + (k == 0 ? 0 : 5) + kind;
}

__device__ __forceinline__ int find_task_problem(const int* __restrict__ base, int nprob, int t) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// MODE 0: integrator pass (epilogue above).  MODE 1: leap-frog step (Sec. 3.1's scheme on
// the 3D system): a.x = level n (cur), a.a = level n-1 (prev, overwritten with level n+1 in
// fields u, w_x, w_y, w_z and psi), a.m = damping variant (0 time-averaged, 1 explicit),
// a.dt; psi^{n+1} = psi^n + dt (u^n + u^{n+1}) / 2.
template <int R, int NW, int NST, int MODE>
__global__ void __launch_bounds__(NW * 32 + 32, 1)
stage_tma3d_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tbase, int nprob,
                   int ntasks, StageArgs a, int* err) {
    using L = Stage3<R>;
    constexpr int NCONS = NW * 32;
    constexpr int NR = L::PL / NCONS;              // consecutive rows per consumer thread
    static_assert(NR * NCONS == L::PL && BY3 % NR == 0, "tile rows must split evenly");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NST];
    __shared__ __align__(8) uint64_t empty[NST];
    __shared__ Info3 info[NST];
    __shared__ int s_err;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], NW);
        }
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const bool has_u = a.u >= 0, has_a = a.a >= 0;
    const uint32_t bytes_warm = 2u * L::PL * 4u;
    // the leap-frog step does not read v
    const uint32_t bytes_full = (uint32_t)(L::PU_OFF * 4) - (MODE == 1 ? L::PL * 4u : 0u) +
                                (has_u ? 6u * L::PL * 4u : 0u) + (has_a ? 6u * L::PL * 4u : 0u);
    int issued = 0;

    if (warp == NW) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int it = 0;
            bool stop = false;
            for (int task = blockIdx.x; task < ntasks && !stop; task += gridDim.x) {
                const int pid = find_task_problem(tbase, nprob, task);
                const ProblemDev* P = probs + pid;
                const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P->tmaps);
                const int tiles_x = (P->nx + BX - 1) / BX;
                const int tiles_y = (P->ny + BY3 - 1) / BY3;
                const int lt = task - __ldg(tbase + pid);
                const int x0 = (lt % tiles_x) * BX;
                const int r = lt / tiles_x;
                const int y0 = (r % tiles_y) * BY3;
                const int k0 = (r / tiles_y) * KC3;
                const int k1 = min(k0 + KC3, P->nz);
                const int kx = a.x, vx = a.x == 0 ? 0 : a.x - 1;
                float* Yp = a.y_out >= 0 ? (a.y_out == 0 ? (float*)P->state
                                                         : (float*)P->work + (long long)(a.y_out - 1) * P->vec_stride)
                                         : nullptr;
                float* Ap = a.acc_out >= 0 ? (a.acc_out == 0 ? (float*)P->state
                                                             : (float*)P->work + (long long)(a.acc_out - 1) * P->vec_stride)
                                           : nullptr;
                const float* Xp = a.x == 0 ? (const float*)P->state
                                           : (const float*)P->work + (long long)(a.x - 1) * P->vec_stride;
                // stages: front planes f = k0 - R .. k1 - 1 + R; compute plane c = f - R >= k0
                for (int f = k0 - R; f < k1 + R; ++f, ++it) {
                    const int s = it % NST;
                    const uint32_t ph = (uint32_t)(it / NST) & 1u;
                    if (!bar_wait(&empty[s], ph ^ 1u)) {
                        s_err = 1;
                        stop = true;
                        break;
                    }
                    const int c = f - R;
                    const bool warm = c < k0;
                    Info3& ti = info[s];
                    ti.Y = Yp;
                    ti.A = Ap;
                    ti.X = Xp;
                    ti.fstr = P->field_stride;
                    ti.ps = (long long)P->ny * P->pitch;
                    ti.x0 = x0;
                    ti.y0 = y0;
                    ti.c = c;
                    ti.warm = warm ? 1 : 0;
                    ti.nx = P->nx;
                    ti.ny = P->ny;
                    ti.nz = P->nz;
                    ti.pitch = P->pitch;
                    ti.pml = P->pml;
                    ti.fs = P->fs;
                    ti.src_i = P->src_i;
                    ti.src_j = P->src_j;
                    ti.src_k = P->src_k;
                    ti.beta0 = P->fbeta0;
                    ti.inv_pml = P->finv_pml;
                    ti.idx1 = P->finv_dx;
                    ti.idx2 = P->finv_dx2;
                    ti.sig = (a.src_slot >= 0 && P->has_src) ? (float)P->sigma[a.src_slot] : 0.f;
                    ti.xs = a.x_scale_slot >= 0 ? (float)P->kry[a.x_scale_slot] : 1.f;
                    float* st = smem + (size_t)s * L::FLOATS;
                    bar_expect_tx(&full[s], warm ? bytes_warm : bytes_full);
                    tma5(st + L::UF_OFF, map3(maps, kx, 3), x0, y0, f, 0, vx, &full[s]);
                    tma5(st + L::WZ_OFF, map3(maps, kx, 3), x0, y0, f - 1, 4, vx, &full[s]);
                    if (!warm) {
                        tma5(st + L::U_OFF, map3(maps, kx, 0), x0 - TX3, y0 - R, c, 0, vx, &full[s]);
                        tma5(st + L::WX_OFF, map3(maps, kx, 1), x0 - TX3, y0, c, 2, vx, &full[s]);
                        tma5(st + L::WY_OFF, map3(maps, kx, 2), x0, y0 - R, c, 3, vx, &full[s]);
                        if (MODE == 0) tma5(st + L::V_OFF, map3(maps, kx, 3), x0, y0, c, 1, vx, &full[s]);
                        tma3(st + L::C2_OFF, maps + 10, x0, y0, c, &full[s]);
                        tma5(st + L::PS_OFF, map3(maps, kx, 3), x0, y0, c, 5, vx, &full[s]);
                        if (has_u)
                            tma5(st + L::PU_OFF, map3(maps, a.u, 4), x0, y0, c, 0, a.u == 0 ? 0 : a.u - 1,
                                 &full[s]);
                        if (has_a)
                            tma5(st + L::PA_OFF, map3(maps, a.a, 4), x0, y0, c, 0, a.a == 0 ? 0 : a.a - 1,
                                 &full[s]);
                    }
                    issued = it + 1;
                }
            }
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int tx = tid & (BX - 1);
        const int ty = tid / BX;                   // rows NR ty .. NR ty + NR - 1
        const int cxs = tx + TX3;
        const float cxf = (float)a.cx, chf = (float)a.ch, cuf = (float)a.cu, ckf = (float)a.ck;
        const float caf = (float)a.ca, cauf = (float)a.cau, cakf = (float)a.cak;
        const float cayf = (float)a.cay, caxf = (float)a.cax;
        float uq[NR][2 * R + 1];
        float wq[NR][2 * R];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
#pragma unroll
            for (int q = 0; q < 2 * R + 1; ++q) uq[r][q] = 0.f;
#pragma unroll
            for (int q = 0; q < 2 * R; ++q) wq[r][q] = 0.f;
        }
        int it = 0;
        bool stop = false;
        for (int task = blockIdx.x; task < ntasks && !stop; task += gridDim.x) {
            // the number of stages of this task is known from its geometry: recompute it
            const int pid = find_task_problem(tbase, nprob, task);
            const ProblemDev* P = probs + pid;
            const float* btab = P->btab;
            const int nbt = P->nbtab;
            const int tiles_x = (P->nx + BX - 1) / BX;
            const int tiles_y = (P->ny + BY3 - 1) / BY3;
            const int lt = task - __ldg(tbase + pid);
            const int k0 = ((lt / tiles_x) / tiles_y) * KC3;
            const int k1 = min(k0 + KC3, P->nz);
            // the horizontal damping of this thread's column and rows is fixed for the task:
            // looked up once, not per plane
            const int ti_ = (lt % tiles_x) * BX + tx;
            const int nxt = P->nx, nyt = P->ny;
            const float bxn_t = bt3(btab, nbt, 2 * min(ti_ + 1, nxt - ti_));
            const float bxh_t = bt3(btab, nbt, min(2 * ti_ + 3, 2 * (nxt - ti_) - 1));
            float byn_t[NR], byh_t[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int tj_ = ((lt / tiles_x) % tiles_y) * BY3 + NR * ty + r;
                byn_t[r] = bt3(btab, nbt, 2 * min(tj_ + 1, nyt - tj_));
                byh_t[r] = bt3(btab, nbt, min(2 * tj_ + 3, 2 * (nyt - tj_) - 1));
            }
            for (int f = k0 - R; f < k1 + R; ++f, ++it) {
                const int s = it % NST;
                const uint32_t ph = (uint32_t)(it / NST) & 1u;
                if (!bar_wait(&full[s], ph)) {
                    s_err = 1;
                    stop = true;
                    break;
                }
                const Info3& ti = info[s];   // field loads on use (a register copy would spill)
                const float* st = smem + (size_t)s * L::FLOATS;
                // push the front values into the queues
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int pt = (NR * ty + r) * BX + tx;
#pragma unroll
                    for (int q = 0; q < 2 * R; ++q) uq[r][q] = uq[r][q + 1];
#pragma unroll
                    for (int q = 0; q < 2 * R - 1; ++q) wq[r][q] = wq[r][q + 1];
                    uq[r][2 * R] = st[L::UF_OFF + pt];
                    wq[r][2 * R - 1] = st[L::WZ_OFF + pt];
                }
                if (!ti.warm) {
                    const int nx = ti.nx, ny = ti.ny, nz = ti.nz, pml = ti.pml, c = ti.c;
                    const bool fs = ti.fs != 0;
                    const float beta0 = ti.beta0, inv_pml = ti.inv_pml, idx1 = ti.idx1, idx2 = ti.idx2;
                    const long long fstr = ti.fstr, ps = ti.ps;
                    const int i = ti.x0 + tx;
                    const float* su = st + L::U_OFF;
                    const float* swx = st + L::WX_OFF;
                    const float* swy = st + L::WY_OFF;
                    const float bxn = bxn_t, bxh = bxh_t;
                    const float bzn = bt3(btab, nbt, 2 * (fs ? nz - c : min(c + 1, nz - c)));
                    const float bzh = bt3(btab, nbt, fs ? 2 * (nz - c) - 1 : min(2 * c + 3, 2 * (nz - c) - 1));
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int ly = NR * ty + r;
                        const int j = ti.y0 + ly;
                        if (i >= nx || j >= ny) continue;
                        const float* urow = su + (ly + R) * L::SW + cxs;
                        const float* wxrow = swx + ly * L::SW + cxs;
                        const float u = uq[r][R];
                        float px[R], py[R], dx[R], dy[R], dwxv[R], dwyv[R];
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            px[q] = urow[q + 1] + urow[-q - 1];
                            py[q] = urow[(q + 1) * L::SW] + urow[-(q + 1) * L::SW];
                            dx[q] = urow[1 + q] - urow[-q];
                            dy[q] = urow[(1 + q) * L::SW] - urow[-q * L::SW];
                            dwxv[q] = wxrow[q] - wxrow[-1 - q];
                            dwyv[q] = swy[(ly + R + q) * BX + tx] - swy[(ly + R - 1 - q) * BX + tx];
                        }
                        const float uxx = ce_tree<R>(u, px), uyy = ce_tree<R>(u, py);
                        const float dux = st_tree<R>(dx), duy = st_tree<R>(dy);
                        const float dwx = st_tree<R>(dwxv), dwy = st_tree<R>(dwyv);
                        float uzz, dwz, duz;
                        const long long oc = (long long)j * ti.pitch + i;
                        if (fs && c < 4) {
                            const float* ucol = ti.X + oc;
                            const float* wcol = ti.X + 4 * fstr + oc;
                            uzz = 0.f;
#pragma unroll
                            for (int q = 0; q < 9; ++q)
                                uzz += g3t_fs[T3_UZZ + c * 9 + q] * (q < nz ? __ldg(ucol + q * ps) : 0.f);
                            dwz = 0.f;
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                dwz += g3t_fs[T3_DWZ + c * 8 + q] * (q < nz - 1 ? __ldg(wcol + q * ps) : 0.f);
                        } else {
                            float pz[R], dwzv[R];
#pragma unroll
                            for (int q = 0; q < R; ++q) {
                                pz[q] = uq[r][R + q + 1] + uq[r][R - q - 1];
                                dwzv[q] = wq[r][R - 1 - q] - wq[r][R + q];
                            }
                            uzz = ce_tree<R>(u, pz);
                            dwz = st_tree<R>(dwzv);
                        }
                        if (fs && c < 3) {
                            const float* ucol = ti.X + oc;
                            duz = 0.f;
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                duz += g3t_fs[T3_UZ + c * 8 + q] * (q < nz ? __ldg(ucol + q * ps) : 0.f);
                        } else {
                            float dz[R];
#pragma unroll
                            for (int q = 0; q < R; ++q) dz[q] = uq[r][R - q] - uq[r][R + 1 + q];
                            duz = st_tree<R>(dz);
                        }
                        const float byn = byn_t[r], byh = byh_t[r];
                        const int pt = ly * BX + tx;
                        const float xwx = wxrow[0];
                        const float xwy = swy[(ly + R) * BX + tx];
                        const float xwz = wq[r][R];
                        const float c2 = st[L::C2_OFF + pt];
                        const float xpsi = st[L::PS_OFF + pt];
                        const bool at_src = i == ti.src_i && j == ti.src_j && c == ti.src_k;
                        const long long o = (long long)c * ps + oc;
                        // psi terms: (product of the other two b's) d_a psi, zero off the edges
                        float gp[3] = {0.f, 0.f, 0.f};
                        {
                            const float pyz = byn * bzn, pxz = bxn * bzn, pxy = bxn * byn;
                            const float* pc = ti.X + 5 * fstr + o;
                            if (pyz != 0.f && i < nx - 1) gp[0] = pyz * dpsi3<R>(pc, 1, i, nx, false) * idx1;
                            if (pxz != 0.f && j < ny - 1) gp[1] = pxz * dpsi3<R>(pc, ti.pitch, j, ny, false) * idx1;
                            if (pxy != 0.f && c < nz - 1) {
                                float d = 0.f;
                                if (fs && c < 3) {
                                    const float* col = ti.X + 5 * fstr + oc;
#pragma unroll
                                    for (int q = 0; q < 8; ++q)
                                        d += g3t_fs[T3_UZ + c * 8 + q] * (q < nz ? __ldg(col + q * ps) : 0.f);
                                } else {
                                    d = dpsi3<R>(pc, ps, c, nz, true);
                                }
                                gp[2] = pxy * d * idx1;
                            }
                        }
                        if constexpr (MODE == 0) {
                            const float xv = st[L::V_OFF + pt];
                            float hv = -(bxn * byn + byn * bzn + bxn * bzn) * u - (bxn + byn + bzn) * xv
                                       - bxn * byn * bzn * xpsi
                                       + c2 * ((uxx + uyy + uzz) * idx2 + (dwx + dwy + dwz) * idx1);
                            if (at_src) hv += ti.sig;
                            const float hwx = (i < nx - 1) ? (byn + bzn - bxh) * dux * idx1 + gp[0] - bxh * xwx : 0.f;
                            const float hwy = (j < ny - 1) ? (bxn + bzn - byh) * duy * idx1 + gp[1] - byh * xwy : 0.f;
                            const float hwz = (c < nz - 1) ? (bxn + byn - bzh) * duz * idx1 + gp[2] - bzh * xwz : 0.f;
                            const float xf[6] = {u, xv, xwx, xwy, xwz, xpsi};
                            const float hf[6] = {xv, hv, hwx, hwy, hwz, u};
                            float* yp = ti.Y ? ti.Y + o : nullptr;
                            float* ap = ti.A ? ti.A + o : nullptr;
#pragma unroll
                            for (int fld = 0; fld < 6; ++fld) {
                                const bool pad = (fld == 2 && i >= nx - 1) || (fld == 3 && j >= ny - 1) ||
                                                 (fld == 4 && c >= nz - 1);
                                const float uval = has_u ? st[L::PU_OFF + fld * L::PL + pt] : 0.f;
                                const float aval = has_a ? st[L::PA_OFF + fld * L::PL + pt] : 0.f;
                                const float kf = cxf * xf[fld] + (chf * ti.xs) * hf[fld];
                                const float yf = pad ? 0.f : (cuf * uval + ckf * kf);
                                if (yp) yp[fld * fstr] = yf;
                                if (ap) ap[fld * fstr] = pad ? 0.f : (caf * aval + cauf * uval + cakf * kf + cayf * yf + caxf * xf[fld]);
                            }
                        } else {
                            const float dt = (float)a.dt;
                            const float inv_dt2 = 1.f / (dt * dt), inv_2dt = 1.f / (2.f * dt);
                            const float bsum = bxn + byn + bzn;
                            float rhs = -(bxn * byn + byn * bzn + bxn * bzn) * u - bxn * byn * bzn * xpsi
                                        + c2 * ((uxx + uyy + uzz) * idx2 + (dwx + dwy + dwz) * idx1);
                            if (at_src) rhs += ti.sig;
                            const float* pm = st + L::PA_OFF + pt;   // level n-1, six fields
                            const float um = pm[0];
                            // fast (2-ulp) division: the step's own error is far larger
                            const float up = __fdividef((2.f * u - um) * inv_dt2 + bsum * um * inv_2dt + rhs,
                                                        inv_dt2 + bsum * inv_2dt);
                            const bool has[3] = {i < nx - 1, j < ny - 1, c < nz - 1};
                            const float bh[3] = {bxh, byh, bzh};
                            const float gco[3] = {byn + bzn - bxh, bxn + bzn - byh, bxn + byn - bzh};
                            const float du[3] = {dux, duy, duz};
                            const float wcur[3] = {xwx, xwy, xwz};
                            float* out = ti.Y + o;
                            out[0] = up;
#pragma unroll
                            for (int a3 = 0; a3 < 3; ++a3) {
                                float wn = 0.f;
                                if (has[a3]) {
                                    const float wm = pm[(2 + a3) * L::PL];
                                    const float g = gco[a3] * du[a3] * idx1 + gp[a3];
                                    wn = a.m == 0 ? __fdividef((1.f - bh[a3] * dt) * wm + 2.f * dt * g, 1.f + bh[a3] * dt)
                                                  : wm + 2.f * dt * (-bh[a3] * wcur[a3] + g);
                                }
                                out[(2 + a3) * fstr] = wn;
                            }
                            out[5 * fstr] = xpsi + 0.5f * dt * (u + up);   // trapezoid rule, psi_t = u
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) bar_arrive(&empty[s]);
            }
        }
    }
    __syncthreads();
    if (s_err) {
        if (warp == NW && lane == 0) {
            for (int k = issued - 1; k >= 0 && k >= issued - NST; --k)
                (void)bar_wait(&full[k % NST], (uint32_t)(k / NST) & 1u);
        }
        if (tid == 0) atomicOr(err, 1);
    }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode3 = nullptr;

int encoder3() {
    if (g_encode3) return 0;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return -1;
    g_encode3 = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return 0;
}

// 5D map over (x, y, z, field, vector) of one buffer (six fields), box (bx, by, 1, bf, 1).
int enc5(CUtensorMap* out, void* base, const ProblemDev& P, int nvec, int bx, int by, int bf) {
    cuuint64_t dims[5] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz, 6, (cuuint64_t)nvec};
    const cuuint64_t ps = (cuuint64_t)P.ny * P.pitch;
    cuuint64_t strides[4] = {(cuuint64_t)P.pitch * 4, ps * 4, (cuuint64_t)P.field_stride * 4,
                             (cuuint64_t)P.vec_stride * 4};
    cuuint32_t box[5] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)bf, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = g_encode3(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int enc3(CUtensorMap* out, const void* base, const ProblemDev& P, int bx, int by) {
    cuuint64_t dims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz};
    cuuint64_t strides[2] = {(cuuint64_t)P.pitch * 4, (cuuint64_t)P.ny * P.pitch * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode3(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int g_sms3 = 0;

template <int R, int NW, int NST, int MODE>
int launch3(const ProblemDev* probs, const int* tbase, int nprob, int ntasks, const StageArgs& a,
            int* err, cudaStream_t s) {
    const size_t smem = (size_t)NST * Stage3<R>::BYTES + 1024;
    static unsigned long long configured = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    if (!(configured >> dev & 1ull)) {
        if (cudaFuncSetAttribute(stage_tma3d_kernel<R, NW, NST, MODE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
        configured |= 1ull << dev;
    }
    if (!g_sms3) {
        cudaDeviceGetAttribute(&g_sms3, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms3 <= 0) g_sms3 = 1;
    }
    const int grid = ntasks < g_sms3 ? ntasks : g_sms3;
    stage_tma3d_kernel<R, NW, NST, MODE><<<grid, NW * 32 + 32, smem, s>>>(probs, tbase, nprob, ntasks, a, err);
    return 0;
}

}  // namespace

int upload_tma3d_tables(const double* fs_uzz, const double* fs_uz, const double* fs_dwz) {
    float f[92];
    for (int i = 0; i < 36; ++i) f[T3_UZZ + i] = (float)fs_uzz[i];
    for (int i = 0; i < 24; ++i) f[T3_UZ + i] = (float)fs_uz[i];
    for (int i = 0; i < 32; ++i) f[T3_DWZ + i] = (float)fs_dwz[i];
    return cudaMemcpyToSymbol(g3t_fs, f, sizeof(f)) == cudaSuccess ? 0 : -1;
}

int tma3d_tasks_of(const ProblemDev& P) {
    return ((P.nx + BX - 1) / BX) * ((P.ny + BY3 - 1) / BY3) * ((P.nz + KC3 - 1) / KC3);
}

// NMAP3 maps per problem: state and workspace, each with the u halo box, the w_x box, the w_y
// box, a one-field plane and a six-field plane; then c^2 (3D).  Sets P.tmaps.
int build_tensor_maps3d(std::vector<ProblemDev>& probs, int R, const std::vector<int>& work_vecs,
                        void** d_maps_inout) {
    if (encoder3() != 0) return -1;
    const int n = (int)probs.size();
    std::vector<CUtensorMap> maps((size_t)n * NMAP3);
    const int SW = BX + 2 * TX3, SH = BY3 + 2 * R;
    const int bxs[5] = {SW, SW, BX, BX, BX};
    const int bys[5] = {SH, BY3, SH, BY3, BY3};
    const int bfs[5] = {1, 1, 1, 1, 6};
    for (int p = 0; p < n; ++p) {
        const ProblemDev& P = probs[p];
        CUtensorMap* m = maps.data() + (size_t)p * NMAP3;
        for (int k = 0; k < 5; ++k) {
            if (enc5(m + k, P.state, P, 1, bxs[k], bys[k], bfs[k]) != 0) return -1;
            void* wb = P.work ? P.work : P.state;
            const int nv = P.work && work_vecs[p] > 0 ? work_vecs[p] : 1;
            if (enc5(m + 5 + k, wb, P, nv, bxs[k], bys[k], bfs[k]) != 0) return -1;
        }
        if (enc3(m + 10, P.c2, P, BX, BY3) != 0) return -1;
    }
    cudaFree(*d_maps_inout);
    *d_maps_inout = nullptr;
    if (cudaMalloc(d_maps_inout, sizeof(CUtensorMap) * maps.size()) != cudaSuccess) return -1;
    if (cudaMemcpy(*d_maps_inout, maps.data(), sizeof(CUtensorMap) * maps.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return -1;
    for (int p = 0; p < n; ++p)
        probs[p].tmaps = static_cast<char*>(*d_maps_inout) + (size_t)p * NMAP3 * sizeof(CUtensorMap);
    return 0;
}

// warps: 16 consumer warps (one row per thread) or 8 (two rows per thread).
int launch_stage_tma3d(int R, int warps, const ProblemDev* probs, const int* tbase, int nprob,
                       int ntasks, const StageArgs& a, int* err, cudaStream_t s) {
    if (ntasks <= 0) return nprob > 0 ? -1 : 0;
    if (warps == 16) {
        if (R == 4) return launch3<4, 16, 4, 0>(probs, tbase, nprob, ntasks, a, err, s);
        if (R == 2) return launch3<2, 16, 4, 0>(probs, tbase, nprob, ntasks, a, err, s);
    } else {
        if (R == 4) return launch3<4, 8, 4, 0>(probs, tbase, nprob, ntasks, a, err, s);
        if (R == 2) return launch3<2, 8, 4, 0>(probs, tbase, nprob, ntasks, a, err, s);
    }
    return -1;
}

int launch_leapfrog_tma3d(int R, int warps, const ProblemDev* probs, const int* tbase, int nprob,
                          int ntasks, int cur, int prev, int variant, double dt, int* err,
                          cudaStream_t s) {
    if (ntasks <= 0) return nprob > 0 ? -1 : 0;
    StageArgs a{};
    a.x = cur;
    a.u = -1;
    a.a = prev;
    a.y_out = prev;
    a.acc_out = -1;
    a.d = -1;
    a.src_slot = 0;
    a.x_scale_slot = -1;
    a.m = variant;
    a.dt = dt;
    if (warps == 16) {
        if (R == 4) return launch3<4, 16, 4, 1>(probs, tbase, nprob, ntasks, a, err, s);
        if (R == 2) return launch3<2, 16, 4, 1>(probs, tbase, nprob, ntasks, a, err, s);
    } else {
        if (R == 4) return launch3<4, 8, 4, 1>(probs, tbase, nprob, ntasks, a, err, s);
        if (R == 2) return launch3<2, 8, 4, 1>(probs, tbase, nprob, ntasks, a, err, s);
    }
    return -1;
}

}  // namespace ewv
