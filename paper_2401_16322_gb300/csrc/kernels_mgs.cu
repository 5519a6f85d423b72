// Modified Gram-Schmidt of one Arnoldi column in one cooperative launch (Sec. 3.2, the inner
// loop of the Krylov listing).
//
// After the product q_{j+1} = dt H~ v_j (its own pass, without a dot), the column's steps
//   h_{k0,j} = <q_{j+1}, v_{k0}>,
//   for k = k0 .. kmax:  q_{j+1} -= h_{k,j} v_k,
//                        h_{k+1,j} = <q_{j+1}, v_{k+1}>  (k < j)  or  h_{j+1,j} = |q_{j+1}|  (k = j)
// (augmented tails included, breakdown test, s_{j+1} and the next source scalar, exactly as
// the finalisation of the flat passes in krylov_finalize.cuh) run in one kernel that keeps
// q_{j+1} in shared memory: the column reads q_{j+1} and each v_k once and writes q_{j+1}
// once, where the flat passes read three vectors and write one per step, and it replaces
// kmax - k0 + 2 launches, each with its own launch latency and serial finalisation, by one.
//
// Layout: block b owns the flat passes' chunks b cpb .. b cpb + cpb - 1 (PCHUNK elements of one
// problem's padded vector each, found through the chunk table), with the same thread-to-element
// mapping, the same per-chunk partial sums and the same fixed-order totals as the flat passes,
// so both forms give the same values bit for bit (FP32; in FP64 the flat form fuses the first
// dot into the stencil pass, another summation order).  Each step's partials go to a buffer of
// their own (two, alternating), a grid barrier makes them visible, and every block sums its
// problems' partials and replays the scalar recurrence on a private copy of tail_{j+1} and of
// column j of H; the block that owns a problem's chunk 0 writes the results back.
//
// The grid must be co-resident (cooperative launch; the host checks the occupancy and
// otherwise runs the flat passes).  Each barrier wait is bounded by the wait limit (1 s, or
// what ewv_debug_set_wait_limit set): on expiry the block sets bit 0 of the error word and
// returns, and the host reports EWV_ERR_TIMEOUT; the arrival counter is cleared before every
// launch.
#include <math.h>

#include "ewave_internal.cuh"
#include "flat_vec.cuh"
#include "krylov_finalize.cuh"

namespace ewv {

__device__ unsigned long long g_mgs_wait_limit_ns = 1000000000ull;

int set_mgs_wait_limit_ns(unsigned long long ns) {
    return cudaMemcpyToSymbol(g_mgs_wait_limit_ns, &ns, sizeof(ns)) == cudaSuccess ? 0 : -1;
}

namespace {

__device__ __forceinline__ unsigned long long mgs_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier over all blocks: bar[0] counts arrivals, bar[1] is the generation.  The
// last block to arrive clears the count and advances the generation; the others wait for it,
// at most limit_ns.  Returns false (in every thread of the block) if the wait gave up.
__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, unsigned long long limit_ns, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned int* gen = bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        bool ok = true;
        if (atomicAdd(bar, 1u) + 1u == nblocks) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else if (limit_ns == 0) {
            ok = false;   // the testing limit: every wait that is not the last arrival gives up
        } else {
            const unsigned long long t0 = mgs_now_ns();
            while (*gen == g) {
                if (mgs_now_ns() - t0 > limit_ns) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Fixed-order total of a problem's partials (the order of partial_and_finalize_at); valid on
// thread 0.
__device__ __forceinline__ double problem_total(const double* partials, int base, int count, double* red,
                                               int tid) {
    double v = 0.0;
    for (int t = tid; t < count; t += NTHREADS) v += __ldcg(partials + base + t);
    return block_sum_fixed(v, red);
}

// (at most 48 registers a thread: five blocks per SM keep one chunk per block co-resident
// up to 760 chunks)
template <typename T>
__global__ void __launch_bounds__(NTHREADS, 5)
mgs_column_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ pbase, int nprob, int nchunks,
                  MgsArgs ma) {
    using V = typename Vec16<T>::type;
    constexpr int NV = Vec16<T>::N;
    constexpr int QPC = PCHUNK / NV;   // 16-byte vectors per chunk
    extern __shared__ __align__(16) unsigned char mgs_smem[];
    V* wsh = reinterpret_cast<V*>(mgs_smem);   // [cpb][QPC]: this block's chunks of q_{j+1}
    __shared__ double red[NTHREADS / 32];
    __shared__ double s_tw[MGS_MAX_CPB][MAX_P];      // tail_{j+1}
    // the step's read-only scalars, loaded before its barrier (the wait hides their latency):
    // two tails (or W) and two slot scales
    __shared__ double s_ta[MGS_MAX_CPB][MAX_P];
    __shared__ double s_tb[MGS_MAX_CPB][MAX_P];
    __shared__ double s_sc[MGS_MAX_CPB][2];
    __shared__ double s_h[MGS_MAX_CPB][MAX_M + 1];   // h_{k,j} at k - 1
    __shared__ int s_act[MGS_MAX_CPB];     // the problem's Arnoldi process goes on
    __shared__ int s_start[MGS_MAX_CPB];   // ... was active when the column started
    __shared__ int s_tail[MGS_MAX_CPB];    // tail_{j+1} was formed (finite first dot)
    __shared__ int s_ok;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int j = ma.j, cpb = ma.cpb;
    const unsigned long long lim = g_mgs_wait_limit_ns;
    const int2* table = reinterpret_cast<const int2*>(pbase + flat_block_table(nprob));

    // per slot: problem, element range, activity; load the chunk of q_{j+1}
    for (int sl = 0; sl < cpb; ++sl) {
        const int g = blockIdx.x * cpb + sl;
        if (g >= nchunks) {
            if (tid == 0) s_act[sl] = s_start[sl] = s_tail[sl] = 0;
            continue;
        }
        const int2 pc = __ldg(table + g);
        const ProblemDev* P = probs + pc.x;
        const bool act = P->kry[KRY_ACTIVE] != 0.0;
        if (tid == 0) {
            s_act[sl] = s_start[sl] = act ? 1 : 0;
            s_tail[sl] = 0;
        }
        if (!act) continue;
        const long long nelem = (long long)P->nfields * P->field_stride;
        const long long e0 = (long long)pc.y * PCHUNK;
        const long long e1 = e0 + PCHUNK < nelem ? e0 + PCHUNK : nelem;
        const long long q0 = e0 / NV, q1 = e1 / NV;
        const V* W = reinterpret_cast<const V*>(vptr<T>(P, j));
        const V* D = reinterpret_cast<const V*>(vptr<T>(P, ma.k0 - 1));
        V* ws = wsh + (size_t)sl * QPC;
        double accd = 0.0;
        for (long long q = q0 + tid; q < q1; q += NTHREADS) {
            const V w = W[q];
            ws[q - q0] = w;
            accd += dotv(w, D[q]);
        }
        const double bsum = block_sum_fixed(accd, red);
        if (tid == 0) ma.partials[g] = bsum;
        double* kry = P->kry;
        if (tid < P->p) {
            s_ta[sl][tid] = kry_tail(kry, j)[tid];
            s_tb[sl][tid] = kry_tail(kry, ma.k0)[tid];
        }
        if (tid == 32) {
            s_sc[sl][0] = kry[KRY_S + j];
            s_sc[sl][1] = kry[KRY_S + ma.k0];
        }
    }
    int buf = 0;
    if (!grid_barrier(ma.bar, gridDim.x, lim, &s_ok)) {
        if (tid == 0) atomicOr(ma.err, 1);
        return;
    }
    // h_{k0,j} and tail_{j+1} = J (s_j tail_j) (FIN_MATVEC)
    for (int sl = 0; sl < cpb; ++sl) {
        if (!s_act[sl]) continue;   // uniform over the block
        const int g = blockIdx.x * cpb + sl;
        const int2 pc = __ldg(table + g);
        const ProblemDev* P = probs + pc.x;
        const double tot = problem_total(ma.partials, g - pc.y, P->pchunks, red, tid);
        if (tid == 0) {
            double* kry = P->kry;
            const bool writer = pc.y == 0;
            const int p = P->p;
            if (!isfinite(tot)) {
                s_act[sl] = 0;
                if (writer) {
                    kry[KRY_NONFINITE] = 1.0;
                    kry[KRY_ACTIVE] = 0.0;
                }
            } else {
                const int k0 = ma.k0;
                const double sj = s_sc[sl][0];
                const double* tj = s_ta[sl];
                const double* tk0 = s_tb[sl];
                double* a = s_tw[sl];
                for (int q = 0; q < p; ++q) a[q] = tj[q];
                for (int q = 0; q < p - 1; ++q) a[q] = sj * a[q + 1];
                a[p - 1] = 0.0;
                double d = 0.0;
                for (int q = 0; q < p; ++q) d += a[q] * tk0[q];
                const double h = s_sc[sl][1] * (tot + d);
                s_h[sl][k0 - 1] = h;
                s_tail[sl] = 1;
                if (writer) kry[KRY_H + (k0 - 1) * MAX_M + (j - 1)] = h;
            }
        }
        __syncthreads();
    }
    // the Gram-Schmidt steps k = k0 .. kmax
    for (int k = ma.k0; k <= ma.kmax; ++k) {
        buf ^= 1;
        double* part = ma.partials + (size_t)buf * nchunks;
        for (int sl = 0; sl < cpb; ++sl) {
            if (!s_act[sl]) continue;
            const int g = blockIdx.x * cpb + sl;
            const int2 pc = __ldg(table + g);
            const ProblemDev* P = probs + pc.x;
            const long long nelem = (long long)P->nfields * P->field_stride;
            const long long e0 = (long long)pc.y * PCHUNK;
            const long long e1 = e0 + PCHUNK < nelem ? e0 + PCHUNK : nelem;
            const long long q0 = e0 / NV, q1 = e1 / NV;
            const T coef = (T)(s_h[sl][k - 1] * P->kry[KRY_S + k]);
            const V* Qk = reinterpret_cast<const V*>(vptr<T>(P, k - 1));
            const V* Qn = k < j ? reinterpret_cast<const V*>(vptr<T>(P, k)) : nullptr;
            V* ws = wsh + (size_t)sl * QPC;
            double accd = 0.0;
#pragma unroll 2
            for (long long q = q0 + tid; q < q1; q += NTHREADS) {
                const V qk = Qk[q];
                const V qn = Qn ? Qn[q] : V{};
                const V w = axpy16(ws[q - q0], coef, qk);
                ws[q - q0] = w;
                accd += dotv(w, Qn ? qn : w);
            }
            const double bsum = block_sum_fixed(accd, red);
            if (tid == 0) part[g] = bsum;
            double* kry = P->kry;
            if (tid < P->p) {
                s_ta[sl][tid] = kry_tail(kry, k)[tid];
                s_tb[sl][tid] = (k < j ? kry_tail(kry, k + 1) : kry + KRY_W)[tid];
            }
            if (tid == 32) {
                s_sc[sl][0] = kry[KRY_S + k];
                s_sc[sl][1] = k < j ? kry[KRY_S + k + 1] : 0.0;
            }
        }
        if (!grid_barrier(ma.bar, gridDim.x, lim, &s_ok)) {
            if (tid == 0) atomicOr(ma.err, 1);
            return;
        }
        // FIN_MGS of step k
        for (int sl = 0; sl < cpb; ++sl) {
            if (!s_act[sl]) continue;
            const int g = blockIdx.x * cpb + sl;
            const int2 pc = __ldg(table + g);
            const ProblemDev* P = probs + pc.x;
            const double tot = problem_total(part, g - pc.y, P->pchunks, red, tid);
            if (tid == 0) {
                double* kry = P->kry;
                const bool writer = pc.y == 0;
                const int p = P->p;
                if (!isfinite(tot)) {
                    s_act[sl] = 0;
                    if (writer) {
                        kry[KRY_NONFINITE] = 1.0;
                        kry[KRY_ACTIVE] = 0.0;
                    }
                } else {
                    const double hkj = s_h[sl][k - 1];
                    const double sk = s_sc[sl][0];
                    const double* tk = s_ta[sl];
                    double* w = s_tw[sl];
                    for (int q = 0; q < p; ++q) w[q] -= hkj * sk * tk[q];
                    if (k < j) {
                        const double* tn = s_tb[sl];
                        double d = 0.0;
                        for (int q = 0; q < p; ++q) d += w[q] * tn[q];
                        const double h = s_sc[sl][1] * (tot + d);
                        s_h[sl][k] = h;
                        if (writer) kry[KRY_H + k * MAX_M + (j - 1)] = h;
                    } else {
                        double d = 0.0;
                        for (int q = 0; q < p; ++q) d += w[q] * w[q];
                        const double h = sqrt(tot + d);
                        if (j < ma.m) {
                            if (writer) kry[KRY_H + j * MAX_M + (j - 1)] = h;
                            if (!(h > ma.tol)) {
                                s_act[sl] = 0;
                                if (writer) {
                                    kry[KRY_ACTIVE] = 0.0;
                                    kry[KRY_MEFF] = (double)j;
                                }
                            } else if (writer) {
                                kry[KRY_S + j + 1] = 1.0 / h;
                                double sg = 0.0;
                                for (int q = 0; q < p; ++q) sg += s_tb[sl][q] * w[q];
                                P->sigma[j + 1] = P->has_src ? sg : 0.0;
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    // write q_{j+1} and tail_{j+1} back (problems active when the column started)
    for (int sl = 0; sl < cpb; ++sl) {
        if (!s_start[sl]) continue;
        const int g = blockIdx.x * cpb + sl;
        const int2 pc = __ldg(table + g);
        const ProblemDev* P = probs + pc.x;
        const long long nelem = (long long)P->nfields * P->field_stride;
        const long long e0 = (long long)pc.y * PCHUNK;
        const long long e1 = e0 + PCHUNK < nelem ? e0 + PCHUNK : nelem;
        const long long q0 = e0 / NV, q1 = e1 / NV;
        V* W = reinterpret_cast<V*>(vptr<T>(P, j));
        const V* ws = wsh + (size_t)sl * QPC;
        for (long long q = q0 + tid; q < q1; q += NTHREADS) W[q] = ws[q - q0];
        if (pc.y == 0 && s_tail[sl] && tid < P->p) kry_tail(P->kry, j + 1)[tid] = s_tw[sl][tid];
    }
}

}  // namespace

int mgs_column_chunks_per_block(int precision, int nchunks) {
    if (nchunks <= 0) return 0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return 0;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    for (int cpb = 1; cpb <= MGS_MAX_CPB; ++cpb) {
        const size_t smem = (size_t)cpb * PCHUNK * (precision == 0 ? sizeof(float) : sizeof(double));
        const void* fn = precision == 0 ? (const void*)mgs_column_kernel<float> : (const void*)mgs_column_kernel<double>;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTHREADS, smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const long long blocks = (nchunks + cpb - 1) / cpb;
        if (blocks <= (long long)per_sm * nsm) return cpb;
    }
    return 0;
}

int launch_mgs_column(int precision, int nchunks, int cpb, const ProblemDev* probs, const int* pbase, int nprob,
                      const MgsArgs& ma_in, cudaStream_t s) {
    if (nchunks <= 0 || cpb < 1 || cpb > MGS_MAX_CPB) return -1;
    MgsArgs ma = ma_in;
    ma.cpb = cpb;
    if (cudaMemsetAsync(ma.bar, 0, sizeof(unsigned int), s) != cudaSuccess) return -1;
    const size_t smem = (size_t)cpb * PCHUNK * (precision == 0 ? sizeof(float) : sizeof(double));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((nchunks + cpb - 1) / cpb));
    cfg.blockDim = dim3(TPX, TPY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = precision == 0
                              ? cudaLaunchKernelEx(&cfg, mgs_column_kernel<float>, probs, pbase, nprob, nchunks, ma)
                              : cudaLaunchKernelEx(&cfg, mgs_column_kernel<double>, probs, pbase, nprob, nchunks, ma);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace ewv
