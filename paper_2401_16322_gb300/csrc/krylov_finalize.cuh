// Arnoldi bookkeeping done by the last-arriving block of a pass (Sec. 3.2, Krylov listing).
//
// Basis vectors are kept unnormalised on the grid: slot k holds q_k and v_k = s_k q_k with
// the scale s_k = 1 / h_{k,k-1} (s_1 = 1/|x|) stored per problem.  The augmented tail of
// each slot (p entries, Eq. matrix_ampli) is stored unscaled beside it.  A pass writes one
// partial dot product per block; the block that arrives last (per-problem atomic counter,
// no waiting) sums the partials in a fixed order -- deterministic -- and runs the scalar
// step below on one thread.  Modes:
//   FIN_NORM0   tot = |u_n|^2      -> tail_1 = eta e_p with eta = |u_n| (1 if u_n = 0) and
//               W scaled by 1/eta (balances the augmented tail against the wavefield; the
//               exact exponential is unchanged), beta = sqrt(tot + eta^2), s_1
//   FIN_MATVEC  tot = <q_{j+1}, q_1> after q_{j+1} = dt H~ v_j
//               -> tail_{j+1} = J (s_j tail_j), h_{1,j}
//   FIN_MGS     pass k of step j: q_{j+1} -= h_{k,j} v_k, tot = <q_{j+1}, q_{k+1}> (k < j)
//               or |q_{j+1}|^2 (k = j) -> h_{k+1,j} or h_{j+1,j}, s_{j+1}, breakdown test
//   FIN_NORM0_TAIL  (adaptive substeps) beta = sqrt(tot + |tail_1|^2) from the tail already
//               in slot 1; problems marked KRY_SKIP stay inactive
//   FIN_STORE_NORM  kry[KRY_AN] = tot (the grid part of |A v_{j+1}|^2 for the error estimate)
// The source contribution of the next matrix-vector product, W . tail_j (unscaled), goes to
// sigma[j].
#pragma once

#include <math.h>

#include "ewave_internal.cuh"

namespace ewv {

enum { FIN_NONE = 0, FIN_NORM0 = 1, FIN_MATVEC = 2, FIN_MGS = 3, FIN_NORM0_NOTAIL = 4,
       FIN_NORM0_TAIL = 5, FIN_STORE_NORM = 6 };

__device__ __forceinline__ double* kry_tail(double* kry, int k) {  // k = 1..MAX_M+1
    return kry + KRY_T + (k - 1) * MAX_P;
}

__device__ inline void krylov_finalize(const ProblemDev* P, int mode, int j, int k, int m,
                                       double tol, double tot) {
    __shared__ double fin_buf[3][MAX_P];   // one thread per block runs this
    double* kry = P->kry;
    const int p = P->p;
    if (!isfinite(tot)) {
        kry[KRY_NONFINITE] = 1.0;
        kry[KRY_ACTIVE] = 0.0;
        return;
    }
    if (mode == FIN_STORE_NORM) {
        kry[KRY_AN] = tot;
        return;
    }
    if (mode == FIN_NORM0_TAIL) {
        // a later substep of the adaptive step: the tail of slot 1 is the previous substep's
        // (uploaded by the host) and W is already scaled by this step's eta; H was zeroed by
        // the finalising block (zero_krylov_start)
        if (kry[KRY_SKIP] != 0.0) {
            kry[KRY_ACTIVE] = 0.0;
            return;
        }
        const double* t1 = kry_tail(kry, 1);
        double tt = 0.0;
        for (int q = 0; q < p; ++q) tt += t1[q] * t1[q];
        const double beta = sqrt(tot + tt);
        kry[KRY_BETA] = beta;
        kry[KRY_S + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
        kry[KRY_ACTIVE] = beta > 0.0 ? 1.0 : 0.0;
        kry[KRY_MEFF] = (double)m;
        double sg = 0.0;
        for (int q = 0; q < p; ++q) sg += kry[KRY_W + q] * t1[q];
        P->sigma[1] = P->has_src ? sg : 0.0;
        return;
    }
    if (mode == FIN_NORM0_NOTAIL) {
        // Arnoldi on a plain (non-augmented) operator, e.g. dt H^T: zero tail, no source (the
        // tails, W, sigma and H were zeroed by the finalising block: zero_krylov_start)
        const double beta = sqrt(tot);
        kry[KRY_BETA] = beta;
        kry[KRY_S + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
        kry[KRY_ACTIVE] = beta > 0.0 ? 1.0 : 0.0;
        kry[KRY_MEFF] = beta > 0.0 ? (double)m : 0.0;
    } else if (mode == FIN_NORM0) {
        double* t1 = kry_tail(kry, 1);
        kry[KRY_SKIP] = 0.0;
        const double eta = tot > 0.0 ? sqrt(tot) : 1.0;
        for (int q = 0; q < MAX_P; ++q) t1[q] = 0.0;
        t1[p - 1] = eta;
        for (int q = 0; q < MAX_P; ++q) kry[KRY_W + q] /= eta;
        const double beta = sqrt(tot + eta * eta);
        kry[KRY_BETA] = beta;
        kry[KRY_S + 1] = 1.0 / beta;
        kry[KRY_ACTIVE] = 1.0;
        kry[KRY_MEFF] = (double)m;
        double sg = 0.0;
        for (int q = 0; q < p; ++q) sg += kry[KRY_W + q] * t1[q];
        P->sigma[1] = P->has_src ? sg : 0.0;
    } else if (mode == FIN_MATVEC) {
        // tot = <q_{j+1}, q_{k0}>, k0 = k (the first vector this step orthogonalises against:
        // 1 for full Gram-Schmidt, j - q + 1 with an orthogonalisation window of q)
        // (the tails are copied to shared memory before any store to them: a load after a
        // store to the same array could not be issued ahead of it, one memory latency per
        // entry; the copies in shared memory cannot alias the global rows)
        const int k0 = k >= 1 ? k : 1;
        const double sj = kry[KRY_S + j];
        const double* tj = kry_tail(kry, j);
        double* tw = kry_tail(kry, j + 1);
        const double* tk0 = kry_tail(kry, k0);
        double* a = fin_buf[0];
        double* b = fin_buf[1];
        for (int q = 0; q < p; ++q) {
            a[q] = tj[q];
            b[q] = tk0[q];
        }
        for (int q = 0; q < p - 1; ++q) a[q] = sj * a[q + 1];   // J (s_j tail_j)
        a[p - 1] = 0.0;
        double d = 0.0;
        for (int q = 0; q < p; ++q) d += a[q] * b[q];
        for (int q = 0; q < p; ++q) tw[q] = a[q];
        kry[KRY_H + (k0 - 1) * MAX_M + (j - 1)] = kry[KRY_S + k0] * (tot + d);
    } else if (mode == FIN_MGS) {
        // loads first, as in FIN_MATVEC; c holds tail_{k+1} (k < j) or W (k = j)
        const double hkj = kry[KRY_H + (k - 1) * MAX_M + (j - 1)];
        const double sk = kry[KRY_S + k];
        const double* tk = kry_tail(kry, k);
        double* tw = kry_tail(kry, j + 1);
        const double* tc = k < j ? kry_tail(kry, k + 1) : kry + KRY_W;
        double* a = fin_buf[0];
        double* w = fin_buf[1];
        double* c = fin_buf[2];
        for (int q = 0; q < p; ++q) {
            a[q] = tk[q];
            w[q] = tw[q];
            c[q] = tc[q];
        }
        for (int q = 0; q < p; ++q) w[q] -= hkj * sk * a[q];
        for (int q = 0; q < p; ++q) tw[q] = w[q];
        if (k < j) {
            double d = 0.0;
            for (int q = 0; q < p; ++q) d += w[q] * c[q];
            kry[KRY_H + k * MAX_M + (j - 1)] = kry[KRY_S + k + 1] * (tot + d);
        } else {
            double d = 0.0;
            for (int q = 0; q < p; ++q) d += w[q] * w[q];
            const double h = sqrt(tot + d);
            if (j < m) {
                kry[KRY_H + j * MAX_M + (j - 1)] = h;
                if (!(h > tol)) {
                    kry[KRY_ACTIVE] = 0.0;
                    kry[KRY_MEFF] = (double)j;
                } else {
                    kry[KRY_S + j + 1] = 1.0 / h;
                    double sg = 0.0;
                    for (int q = 0; q < p; ++q) sg += c[q] * w[q];
                    P->sigma[j + 1] = P->has_src ? sg : 0.0;
                }
            }
        }
    }
}

// Block-wide fixed-order sum of one double per thread (blockDim.x * blockDim.y == NTHREADS).
__device__ __forceinline__ double block_sum_fixed(double v, double* red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0) {
        for (int w = 0; w < NTHREADS / 32; ++w) s += red[w];
    }
    __syncthreads();
    return s;   // valid on thread 0
}

// The zeroing that starts an Arnoldi process (modes FIN_NORM0*), spread over the finalising
// block: the Hessenberg block, and for FIN_NORM0_NOTAIL every tail, W and sigma.  Called by
// all threads; ends with a barrier.
__device__ inline void zero_krylov_start(const ProblemDev* P, int mode, int tid) {
    if (mode != FIN_NORM0 && mode != FIN_NORM0_NOTAIL && mode != FIN_NORM0_TAIL) return;
    double* kry = P->kry;
    for (int r = tid; r < (MAX_M + 1) * MAX_M; r += NTHREADS) kry[KRY_H + r] = 0.0;
    if (mode == FIN_NORM0_NOTAIL) {
        for (int r = tid; r < (MAX_M + 1) * MAX_P; r += NTHREADS) kry[KRY_T + r] = 0.0;
        for (int r = tid; r < MAX_P; r += NTHREADS) kry[KRY_W + r] = 0.0;
        for (int r = tid; r <= MAX_M; r += NTHREADS) P->sigma[r] = 0.0;
    }
    __syncthreads();
}

// Write this block's partial into slot `slot`; if it is the last of the problem's `count`
// blocks (slots base .. base + count - 1), sum all partials in a fixed order and finalise.
// Must be called by all threads of the block.
__device__ inline void partial_and_finalize_at(const ProblemDev* P, int pid, const StageArgs& a,
                                               double block_partial_on_t0, double* red,
                                               int* s_last, int slot, int base, int count) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid == 0) {
        a.partials[slot] = block_partial_on_t0;
        __threadfence();
        const unsigned int prev = atomicAdd(a.counters + pid, 1u);
        *s_last = (prev == (unsigned int)(count - 1));
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    double v = 0.0;
    for (int t = tid; t < count; t += NTHREADS) v += __ldcg(a.partials + base + t);
    const double tot = block_sum_fixed(v, red);
    zero_krylov_start(P, a.fin_mode, tid);
    if (tid == 0) {
        krylov_finalize(P, a.fin_mode, a.fin_j, a.fin_k, a.m, a.tol, tot);
        a.counters[pid] = 0u;
        __threadfence();
    }
}

// The tile-list form: one block per tile, slot = block index.
__device__ inline void partial_and_finalize(const ProblemDev* P, int pid, const StageArgs& a,
                                            double block_partial_on_t0, double* red,
                                            int* s_last) {
    partial_and_finalize_at(P, pid, a, block_partial_on_t0, red, s_last, blockIdx.x,
                            P->tile_base, P->ntiles);
}

}  // namespace ewv
