// Small and pointwise kernels around the fused stencil passes:
//  - step clock and per-step source scalars (Ricker derivatives, augmented tail recurrence)
//  - receiver recording (seismogram, Sec. 5.1)
//  - Krylov passes: |x|^2, modified Gram-Schmidt axpy + next dot (Sec. 3.2 listing), the
//    final combination, and the [13/13] Pade exponential of the Hessenberg matrix
//  - Faber coefficients by the trapezoid rule on the unit circle (FP64)
//  - vector copy / swap helpers
#include <math.h>

#include "ewave_internal.cuh"
#include "flat_vec.cuh"
#include "krylov_finalize.cuh"

namespace ewv {

// ---------------------------------------------------------------- clock
__global__ void set_clock_kernel(const ProblemDev* probs, int nprob, double t, double dt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    const ProblemDev* P = probs + p;
    P->clk[0] = 0;
    P->tclk[0] = t;
    P->tclk[1] = dt;
    P->kry[KRY_NONFINITE] = 0.0;   // the flag reports non-finite values within one call
}

__global__ void reset_cursor_kernel(const ProblemDev* probs, int nprob) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    probs[p].clk[1] = 0;
}

// ---------------------------------------------------------------- source scalars
// Ricker r(tau) = (1 - 2 a tau^2) exp(-a tau^2), a = (pi f)^2 (Sec. 4.1).  Its derivatives
// (prologue_kernel) follow r^(k) = -g^(k+2) / (2a), g = exp(-a tau^2), with the Hermite
// recurrence g^(k) = -2 a tau g^(k-1) - 2 a (k-1) g^(k-2).
__device__ __forceinline__ double ricker(double t, double f, double t0) {
    const double a = (M_PI * f) * (M_PI * f);
    const double tau = t - t0;
    return (1.0 - 2.0 * a * tau * tau) * exp(-a * tau * tau);
}

enum { PRO_FABER = 1, PRO_KRYLOV = 2, PRO_HORK = 3, PRO_RK32 = 4, PRO_RK44 = 5, PRO_LEAPFROG = 6,
       PRO_HORK_HORNER = 7 };

// One warp per problem.  Fills sigma[] (the value added at the source node's v entry in
// each pass of this step) from t_n = t_start + step * dt:
//   Faber: sigma_j = W . y_j, y_0 = e_p, y_1 = F1 y_0, y_2 = F1 y_1 - 2 c1 y_0,
//          y_j = F1 y_{j-1} - c1 y_{j-2}, F1 = (J/dt)/gamma - c0 (tail of Eq. matrix_ampli)
//   HORK:  sigma_i = W . (I + J)^i e_p
//   HORK in Horner form (passes j = m .. 1): sigma_k = W . y_{j+1} with j = m - k,
//          y_{m+1} = e_p, y_j = e_p + (1/j) J y_{j+1}
//   RK3-2 / RK4-4 / leap-frog: f at the stage times
//   Krylov: W stored for the Arnoldi passes
// W[p-1-k] = dt^k r^(k)(t_n) amp / dx^2 (tail scaled by dt).  Lane q holds tail entry q;
// the shift J (J y)_q = y_{q+1} is a warp shuffle, each W . y a warp reduction.
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void prologue_kernel(const ProblemDev* probs, int nprob, int kind, int m,
                                double gamma, double c0, double c1) {
    const int pid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int q = threadIdx.x & 31;
    if (pid >= nprob) return;           // whole warps exit together
    const ProblemDev* P = probs + pid;
    const double dt = P->tclk[1];
    const double tn = P->tclk[0] + (double)P->clk[0] * dt;
    double* sg = P->sigma;
    if (!P->has_src) {
        for (int s = q; s < MAX_SIGMA; s += 32) sg[s] = 0.0;
        if (kind == PRO_KRYLOV && q < MAX_P) P->kry[KRY_W + q] = 0.0;
        return;
    }
    const double scale = P->amp * P->inv_dx2;
    if (kind == PRO_RK32 || kind == PRO_RK44 || kind == PRO_LEAPFROG) {
        if (q == 0) {
            if (kind == PRO_LEAPFROG) {
                sg[0] = scale * ricker(tn, P->f_peak, P->t0);
            } else {
                sg[0] = scale * ricker(tn, P->f_peak, P->t0);
                sg[1] = sg[2] = scale * ricker(tn + 0.5 * dt, P->f_peak, P->t0);
                if (kind == PRO_RK44) sg[3] = scale * ricker(tn + dt, P->f_peak, P->t0);
            }
        }
        return;
    }
    const int p = P->p;
    // W_q = dt^k r^(k)(t_n) scale with k = p-1-q: every lane runs the Hermite recurrence
    // g^(k) = -2 a tau g^(k-1) - 2 a (k-1) g^(k-2) and keeps its own term.
    const int kq = p - 1 - q;
    const double a = (M_PI * P->f_peak) * (M_PI * P->f_peak);
    const double tau = tn - P->t0;
    double gm2 = exp(-a * tau * tau), gm1 = -2.0 * a * tau * gm2, rk = 0.0, dk = 1.0;
    for (int k = 2; k < p + 2; ++k) {
        const double g = -2.0 * a * tau * gm1 - 2.0 * a * (double)(k - 1) * gm2;
        if (k - 2 == kq) rk = -g / (2.0 * a);
        gm2 = gm1;
        gm1 = g;
    }
    for (int k = 0; k < kq && kq >= 0; ++k) dk *= dt;
    const double W = (q < p) ? dk * rk * scale : 0.0;
    if (kind == PRO_KRYLOV) {
        if (q < MAX_P) P->kry[KRY_W + q] = W;
        return;
    }
    double y0 = (q == p - 1) ? 1.0 : 0.0;
    if (kind == PRO_HORK_HORNER) {
        double y = y0;
        for (int k = 0; k < m && k < MAX_SIGMA; ++k) {
            const double s = warp_sum(W * y);
            if (q == 0) sg[k] = s;
            double up = __shfl_down_sync(0xffffffffu, y, 1);
            if (q + 1 >= p) up = 0.0;
            y = ((q == p - 1) ? 1.0 : 0.0) + up / (double)(m - k);
        }
        return;
    }
    if (kind == PRO_HORK) {
        // y_i = (I + J) y_{i-1}
        for (int i = 0; i < m && i < MAX_SIGMA; ++i) {
            const double s = warp_sum(W * y0);
            if (q == 0) sg[i] = s;
            double up = __shfl_down_sync(0xffffffffu, y0, 1);
            if (q + 1 >= p) up = 0.0;
            y0 = y0 + up;
        }
        return;
    }
    // Faber
    const double ig = 1.0 / gamma;
    auto F1 = [&](double y) {
        double up = __shfl_down_sync(0xffffffffu, y, 1);
        if (q + 1 >= p) up = 0.0;
        return ig * up / dt - c0 * y;
    };
    double s0 = warp_sum(W * y0);
    if (q == 0) sg[0] = s0;
    double y1 = F1(y0);
    if (m >= 2) {
        const double s1 = warp_sum(W * y1);
        if (q == 0) sg[1] = s1;
    }
    for (int j = 2; j < m && j < MAX_SIGMA; ++j) {
        const double cj = (j == 2) ? 2.0 * c1 : c1;
        const double y2 = F1(y1) - cj * y0;
        const double sj = warp_sum(W * y2);
        if (q == 0) sg[j] = sj;
        y0 = y1;
        y1 = y2;
    }
}

// ---------------------------------------------------------------- recording
template <typename T>
__global__ void record_kernel(const ProblemDev* probs, int nprob, int vec) {
    const ProblemDev* P = probs + blockIdx.x;
    const long long cur = P->clk[1];
    if (P->seismo && cur < P->capacity) {
        const T* u = vptr<T>(P, vec);
        T* out = (T*)P->seismo + cur * P->rec_stride;
        for (int r = threadIdx.x; r < P->nrec; r += blockDim.x) out[r] = u[P->rec_off[r]];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        P->clk[1] = cur + 1;
        P->clk[0] += 1;
    }
}

// ---------------------------------------------------------------- adjoint source
// lambda_u[rec] += values[shot][rec] (the transpose of recording, R^T r); one thread per
// shot adds its receivers in order, so coincident receivers are summed deterministically.
template <typename T>
__global__ void inject_kernel(T* adj, long long vec_elems, const T* values, const int* rec_off,
                              const int* nrec, int nshots, int max_rec) {
    const int sh = blockIdx.x * blockDim.x + threadIdx.x;
    if (sh >= nshots) return;
    T* lam = adj + (long long)sh * vec_elems;
    const int n = nrec[sh];
    for (int r = 0; r < n; ++r) lam[rec_off[sh * max_rec + r]] += values[(long long)sh * max_rec + r];
}

// out[o] = sum_s in[s][o], shots summed in index order (deterministic).
template <typename T>
__global__ void sum_shots_kernel(const T* in, T* out, long long n, int nshots) {
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
         o += (long long)gridDim.x * blockDim.x) {
        T acc = T(0);
        for (int s = 0; s < nshots; ++s) acc += in[(long long)s * n + o];
        out[o] = acc;
    }
}

// ---------------------------------------------------------------- pointwise Krylov passes
// Each uses the stencil kernels' tile decomposition so that partial index == block index.

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
point_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tile_prob,
             PointArgs pa) {
    __shared__ double red[NTHREADS / 32];
    __shared__ int s_last;
    const int pid = tile_prob[blockIdx.x];
    const ProblemDev* P = probs + pid;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = P->nx, ny = P->ny, pitch = P->pitch;
    const int lt = blockIdx.x - P->tile_base;
    // tile (x, y[, z chunk of KC3 planes]); 2D problems have nz = 1 and one z tile
    const int nz = P->nz > 1 ? P->nz : 1;
    const int nf = P->nfields;   // 4 (2D) or 6 (3D: w_z and psi added)
    const int rr = lt / P->tiles_x;
    const int x0 = (lt % P->tiles_x) * BX, y0 = (rr % P->tiles_y) * BY;
    const int k0 = nz > 1 ? (rr / P->tiles_y) * KC3 : 0;
    const int k1 = nz > 1 ? min(k0 + KC3, nz) : 1;
    const long long ps = (long long)ny * pitch;
    const long long fstr = P->field_stride;
    double* kry = P->kry;

    if (pa.mode == 1 && kry[KRY_ACTIVE] == 0.0) return;
    if (pa.mode == 3 || pa.mode == 4 || pa.mode == 6) {
        T* S = vptr<T>(P, pa.mode == 6 ? pa.dst : pa.src);
        T* Dd = vptr<T>(P, pa.dst);
        for (int kz = k0; kz < k1; ++kz)
        for (int b = 0; b < VY; ++b)
            for (int c = 0; c < VX; ++c) {
                const int i = x0 + tx + c * TPX, j = y0 + ty + b * TPY;
                if (i >= nx || j >= ny) continue;
                const long long o = kz * ps + (long long)j * pitch + i;
                for (int f = 0; f < nf; ++f) {
                    if (!((pa.fmask >> f) & 1)) continue;
                    if (pa.mode == 6) {
                        Dd[f * fstr + o] = T(0);
                        continue;
                    }
                    const T s = S[f * fstr + o];
                    if (pa.mode == 4) S[f * fstr + o] = Dd[f * fstr + o];
                    Dd[f * fstr + o] = s;
                }
            }
        return;
    }
    if (pa.mode == 2) {
        // u^{n+1} = beta sum_{k=1}^{meff} e_k s_k q_k  (q_1 is the state itself)
        if (kry[KRY_NONFINITE] != 0.0) return;
        const int meff = (int)kry[KRY_MEFF];
        const double beta = kry[KRY_BETA];
        T coef[MAX_M];
        for (int k = 1; k <= meff; ++k) coef[k - 1] = (T)(beta * kry[KRY_E + k - 1] * kry[KRY_S + k]);
        T* St = vptr<T>(P, 0);
        for (int kz = k0; kz < k1; ++kz)
        for (int b = 0; b < VY; ++b)
            for (int c = 0; c < VX; ++c) {
                const int i = x0 + tx + c * TPX, j = y0 + ty + b * TPY;
                if (i >= nx || j >= ny) continue;
                const long long o = kz * ps + (long long)j * pitch + i;
                for (int f = 0; f < nf; ++f) {
                    T acc = T(0);
                    for (int k = 1; k <= meff; ++k) acc += coef[k - 1] * vptr<T>(P, k - 1)[f * fstr + o];
                    St[f * fstr + o] = acc;
                }
            }
        return;
    }
    // mode 0 (norm of the state) or 1 (MGS pass k of Arnoldi step j):
    // q_{j+1} -= h_{k,j} s_k q_k, then partial <q_{j+1}, q_{k+1}> (k < j) or |q_{j+1}|^2.
    float accf = 0.f;
    double accd = 0.0;
    T* W = nullptr;
    const T* Qk = nullptr;
    const T* Qn = nullptr;
    T coef = T(0);
    if (pa.mode == 0) {
        Qn = vptr<T>(P, 0);
    } else {
        W = vptr<T>(P, pa.j);                  // slot j+1
        Qk = vptr<T>(P, pa.k - 1);             // slot k
        coef = (T)(kry[KRY_H + (pa.k - 1) * MAX_M + (pa.j - 1)] * kry[KRY_S + pa.k]);
        Qn = pa.k < pa.j ? vptr<T>(P, pa.k) : nullptr;   // slot k+1 (or w itself)
    }
    for (int kz = k0; kz < k1; ++kz)
    for (int b = 0; b < VY; ++b)
        for (int c = 0; c < VX; ++c) {
            const int i = x0 + tx + c * TPX, j = y0 + ty + b * TPY;
            if (i >= nx || j >= ny) continue;
            const long long o = kz * ps + (long long)j * pitch + i;
            for (int f = 0; f < nf; ++f) {
                if ((f == 2 && i >= nx - 1) || (f == 3 && j >= ny - 1) || (f == 4 && kz >= nz - 1))
                    continue;
                T val;
                T other;
                if (pa.mode == 0) {
                    val = Qn[f * fstr + o];
                    other = val;
                } else {
                    val = W[f * fstr + o] - coef * Qk[f * fstr + o];
                    W[f * fstr + o] = val;
                    other = Qn ? Qn[f * fstr + o] : val;
                }
                if (sizeof(T) == 4) accf = fmaf((float)val, (float)other, accf);
                else accd = fma((double)val, (double)other, accd);
            }
        }
    if (pa.mode == 1 && pa.k == pa.j && pa.j == pa.m) return;   // h_{m+1,m} unused
    const double bsum = block_sum_fixed((double)accf + accd, red);
    StageArgs a{};
    a.fin_mode = pa.mode == 0 ? FIN_NORM0 : FIN_MGS;
    a.fin_j = pa.j;
    a.fin_k = pa.k;
    a.m = pa.m;
    a.tol = pa.tol;
    a.partials = pa.partials;
    a.counters = pa.counters;
    partial_and_finalize(P, pid, a, bsum, red, &s_last);
}

// ---------------------------------------------------------------- flat pointwise passes
// Modes 0 (|q_1|^2), 1 (MGS pass) and 2 (Krylov combine) over whole padded vectors: every
// pad element is zero in every vector, so the flat sums and updates equal the masked ones.
// Block b handles elements [c PCHUNK, (c + 1) PCHUNK) of problem p ((p, c) from the block
// table after the prefix sums), with
// 16-byte vector loads; its partial dot product goes to slot b, and the problem's last block
// sums the partials in a fixed order (deterministic, no waiting).
__device__ __forceinline__ int flat_problem(const int* __restrict__ base, int nprob, int b) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
point_flat_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ pbase, int nprob,
                  PointArgs pa) {
    using V = typename Vec16<T>::type;
    constexpr int NV = Vec16<T>::N;
    __shared__ double red[NTHREADS / 32];
    __shared__ int s_last;
    __shared__ T s_coef[MAX_M];
    const int2 pc = __ldg(reinterpret_cast<const int2*>(pbase + flat_block_table(nprob)) + blockIdx.x);
    const int pid = pc.x;
    const ProblemDev* P = probs + pid;
    double* kry = P->kry;
    if ((pa.mode == 1 || pa.mode == 5) && kry[KRY_ACTIVE] == 0.0) return;
    if (pa.mode == 2 && (kry[KRY_NONFINITE] != 0.0 || kry[KRY_SKIP] != 0.0)) return;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nf = P->nfields;   // 4 (2D) or 6 (3D: w_z and psi added)
    const long long nelem = (long long)nf * P->field_stride;
    const long long e0 = (long long)pc.y * PCHUNK;
    const long long e1 = e0 + PCHUNK < nelem ? e0 + PCHUNK : nelem;
    const long long q0 = e0 / NV, q1 = e1 / NV;
    if (pa.mode == 2) {
        // u^{n+1} = beta sum_{k=1}^{meff} e_k s_k q_k  (q_1 is the state itself)
        const int meff = (int)kry[KRY_MEFF];
        const double beta = kry[KRY_BETA];
        for (int k = tid; k < meff; k += NTHREADS) s_coef[k] = (T)(beta * kry[KRY_E + k] * kry[KRY_S + k + 1]);
        __syncthreads();
        V* St = pa.out ? reinterpret_cast<V*>(static_cast<T*>(pa.out) + (long long)pid * pa.out_stride)
                       : reinterpret_cast<V*>(vptr<T>(P, pa.dst));
        for (long long q = q0 + tid; q < q1; q += NTHREADS) {
            V acc = {};
            for (int k = 1; k <= meff; ++k) fma16(acc, s_coef[k - 1], reinterpret_cast<const V*>(vptr<T>(P, k - 1))[q]);
            St[q] = acc;
        }
        return;
    }
    double accd = 0.0;
    if (pa.mode == 0) {
        const V* Q = reinterpret_cast<const V*>(vptr<T>(P, 0));
        for (long long q = q0 + tid; q < q1; q += NTHREADS) {
            const V a = Q[q];
            accd += dotv(a, a);
        }
    } else if (pa.mode == 7) {
        const V* W = reinterpret_cast<const V*>(vptr<T>(P, pa.j));      // slot j+1
        for (long long q = q0 + tid; q < q1; q += NTHREADS) {
            const V w = W[q];
            accd += dotv(w, w);
        }
    } else if (pa.mode == 5) {
        // <q_{j+1}, q_k> after the matrix-vector product (its finalisation is FIN_MATVEC)
        const V* W = reinterpret_cast<const V*>(vptr<T>(P, pa.j));      // slot j+1
        const V* D = reinterpret_cast<const V*>(vptr<T>(P, pa.k - 1));  // slot k
        for (long long q = q0 + tid; q < q1; q += NTHREADS) accd += dotv(W[q], D[q]);
    } else {
        V* W = reinterpret_cast<V*>(vptr<T>(P, pa.j));                  // slot j+1
        const V* Qk = reinterpret_cast<const V*>(vptr<T>(P, pa.k - 1));   // slot k
        const V* Qn = pa.k < pa.j ? reinterpret_cast<const V*>(vptr<T>(P, pa.k)) : nullptr;
        const T coef = (T)(kry[KRY_H + (pa.k - 1) * MAX_M + (pa.j - 1)] * kry[KRY_S + pa.k]);
#pragma unroll 2
        for (long long q = q0 + tid; q < q1; q += NTHREADS) {
            const V wq = W[q], qk = Qk[q];
            // every operand is loaded before the store: the loads may not move past a store
            // the compiler cannot prove disjoint, which would cost a second memory round trip
            const V qn = Qn ? Qn[q] : V{};
            const V w = axpy16(wq, coef, qk);
            W[q] = w;
            accd += dotv(w, Qn ? qn : w);
        }
    }
    if (pa.mode == 1 && pa.k == pa.j && pa.j == pa.m) return;   // h_{m+1,m} unused
    const double bsum = block_sum_fixed(accd, red);
    StageArgs a{};
    a.fin_mode = pa.mode == 0 ? (pa.notail == 2 ? FIN_NORM0_TAIL : pa.notail ? FIN_NORM0_NOTAIL : FIN_NORM0)
               : pa.mode == 7 ? FIN_STORE_NORM
               : (pa.mode == 5 ? FIN_MATVEC : FIN_MGS);
    a.fin_j = pa.j;
    a.fin_k = pa.k;
    a.m = pa.m;
    a.tol = pa.tol;
    a.partials = pa.partials;
    a.counters = pa.counters;
    partial_and_finalize_at(P, pid, a, bsum, red, &s_last, blockIdx.x, blockIdx.x - pc.y, P->pchunks);
}

// Multi-output Krylov combine (PointArgs mode 8): output q = beta sum_{k=1}^{meff} e_{q,k} s_k q_k
// for every q from one read of the basis (each output's arithmetic is that of mode 2, so an
// output equals the single combine with the same coefficients bit for bit).  A kernel of its
// own keeps the accumulators out of the flat passes' register budget.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
combine_multi_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ pbase, int nprob, PointArgs pa) {
    using V = typename Vec16<T>::type;
    constexpr int NV = Vec16<T>::N;
    __shared__ T s_mc[MAX_TAU][MAX_M];
    const int2 pc = __ldg(reinterpret_cast<const int2*>(pbase + flat_block_table(nprob)) + blockIdx.x);
    const int pid = pc.x;
    const ProblemDev* P = probs + pid;
    const double* kry = P->kry;
    if (kry[KRY_NONFINITE] != 0.0 || kry[KRY_SKIP] != 0.0) return;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int meff = (int)kry[KRY_MEFF];
    const double beta = kry[KRY_BETA];
    const int nt = pa.nout + pa.final_out;
    const double* ec = pa.ecoef + (size_t)pid * nt * MAX_M;
    for (int e = tid; e < nt * meff; e += NTHREADS) {
        const int q = e / meff, k = e - q * meff;
        s_mc[q][k] = (T)(beta * ec[q * MAX_M + k] * kry[KRY_S + k + 1]);
    }
    __syncthreads();
    const long long nelem = (long long)P->nfields * P->field_stride;
    const long long e0 = (long long)pc.y * PCHUNK;
    const long long e1 = e0 + PCHUNK < nelem ? e0 + PCHUNK : nelem;
    const long long q0 = e0 / NV, q1 = e1 / NV;
    V* outs[MAX_TAU];
#pragma unroll
    for (int q = 0; q < MAX_TAU; ++q) {
        outs[q] = nullptr;
        if (q < pa.nout)
            outs[q] = pa.out ? reinterpret_cast<V*>(static_cast<T*>(pa.out) + q * pa.out_qstride +
                                                    (long long)pid * pa.out_stride)
                             : reinterpret_cast<V*>(vptr<T>(P, pa.dst + q));
        else if (q == pa.nout && pa.final_out)
            outs[q] = reinterpret_cast<V*>(vptr<T>(P, 0));
    }
    for (long long i = q0 + tid; i < q1; i += NTHREADS) {
        V acc[MAX_TAU];
#pragma unroll
        for (int q = 0; q < MAX_TAU; ++q) acc[q] = V{};
        for (int k = 1; k <= meff; ++k) {
            const V v = reinterpret_cast<const V*>(vptr<T>(P, k - 1))[i];
#pragma unroll
            for (int q = 0; q < MAX_TAU; ++q)
                if (q < nt) fma16(acc[q], s_mc[q][k - 1], v);
        }
#pragma unroll
        for (int q = 0; q < MAX_TAU; ++q)
            if (q < nt) outs[q][i] = acc[q];
    }
}

// ---------------------------------------------------------------- Hessenberg exponential
// [13/13] Pade approximant with scaling and squaring (Higham 2005), FP64, one block per
// problem; writes exp(H_meff) e_1 to kry[KRY_E..].  Shared memory: 7 matrices of meff^2.
__device__ void mat_mul(const double* A, const double* B, double* C, int n) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s = fma(A[r * n + k], B[k * n + c], s);
        C[e] = s;
    }
    __syncthreads();
}

// Block (p, q) writes exp(tau_q H_meff) e_1 of problem p to kry[KRY_E..] (et.out null, one
// tau) or to et.out[(p ntau + q) MAX_M ..] (several taus in one launch).
__global__ void expm_kernel(const ProblemDev* probs, int nprob, ExpmTaus et) {
    extern __shared__ double sm[];
    __shared__ double b[14];
    __shared__ double colmax[MAX_M];
    __shared__ int s_scale, s_piv;
    const ProblemDev* P = probs + blockIdx.x;
    double* kry = P->kry;
    const double hscale = et.tau[blockIdx.y];
    double* eo = et.out ? et.out + ((size_t)blockIdx.x * et.n + blockIdx.y) * MAX_M : kry + KRY_E;
    const int n = (int)kry[KRY_MEFF];
    if (n <= 0 || kry[KRY_NONFINITE] != 0.0) return;
    const int nn = n * n;
    double* A = sm;
    double* A2 = A + nn;
    double* A4 = A2 + nn;
    double* A6 = A4 + nn;
    double* Um = A6 + nn;
    double* Vm = Um + nn;
    double* Tm = Vm + nn;
    const int tid = threadIdx.x;
    if (tid == 0) {
        // b_k = (26-k)! 13! / (26! k! (13-k)!)
        double f[27];
        f[0] = 1.0;
        for (int i = 1; i <= 26; ++i) f[i] = f[i - 1] * (double)i;
        for (int k = 0; k <= 13; ++k) b[k] = f[26 - k] * f[13] / (f[26] * f[k] * f[13 - k]);
    }
    for (int e = tid; e < nn; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        A[e] = hscale * kry[KRY_H + r * MAX_M + c];   // exp(tau H_m): dense output at tau
    }
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += fabs(A[r * n + c]);
        colmax[c] = s;
    }
    __syncthreads();
    if (tid == 0) {
        double nrm = 0.0;
        for (int c = 0; c < n; ++c) nrm = fmax(nrm, colmax[c]);
        const double theta13 = 5.371920351148152;
        int s = 0;
        if (nrm > theta13) s = (int)ceil(log2(nrm / theta13));
        s_scale = s;
    }
    __syncthreads();
    const int s = s_scale;
    const double sc = ldexp(1.0, -s);
    for (int e = tid; e < nn; e += blockDim.x) A[e] *= sc;
    __syncthreads();
    mat_mul(A, A, A2, n);
    mat_mul(A2, A2, A4, n);
    mat_mul(A4, A2, A6, n);
    for (int e = tid; e < nn; e += blockDim.x) Tm[e] = b[13] * A6[e] + b[11] * A4[e] + b[9] * A2[e];
    __syncthreads();
    mat_mul(A6, Tm, Um, n);   // Um = A6 (b13 A6 + b11 A4 + b9 A2)
    for (int e = tid; e < nn; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        Tm[e] = Um[e] + b[7] * A6[e] + b[5] * A4[e] + b[3] * A2[e] + (r == c ? b[1] : 0.0);
    }
    __syncthreads();
    mat_mul(A, Tm, Um, n);    // U = A (...)
    for (int e = tid; e < nn; e += blockDim.x) Tm[e] = b[12] * A6[e] + b[10] * A4[e] + b[8] * A2[e];
    __syncthreads();
    mat_mul(A6, Tm, Vm, n);
    for (int e = tid; e < nn; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        Vm[e] += b[6] * A6[e] + b[4] * A4[e] + b[2] * A2[e] + (r == c ? b[0] : 0.0);
    }
    __syncthreads();
    // Solve (V - U) Rm = (V + U): LU with partial pivoting; P_ in A, RHS in A2.
    double* Pm = A;
    double* Q = A2;
    for (int e = tid; e < nn; e += blockDim.x) {
        Pm[e] = Vm[e] - Um[e];
        Q[e] = Vm[e] + Um[e];
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        if (tid == 0) {
            int piv = c;
            double best = fabs(Pm[c * n + c]);
            for (int r = c + 1; r < n; ++r)
                if (fabs(Pm[r * n + c]) > best) {
                    best = fabs(Pm[r * n + c]);
                    piv = r;
                }
            s_piv = piv;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != c) {
            for (int e = tid; e < n; e += blockDim.x) {
                double t = Pm[c * n + e];
                Pm[c * n + e] = Pm[piv * n + e];
                Pm[piv * n + e] = t;
                t = Q[c * n + e];
                Q[c * n + e] = Q[piv * n + e];
                Q[piv * n + e] = t;
            }
        }
        __syncthreads();
        const double d = Pm[c * n + c];
        // eliminate rows below
        for (int e = tid; e < (n - c - 1) * n; e += blockDim.x) {
            const int r = c + 1 + e / n, col = e % n;
            const double l = Pm[r * n + c] / d;
            if (col > c) Pm[r * n + col] -= l * Pm[c * n + col];
            Q[r * n + col] -= l * Q[c * n + col];
        }
        __syncthreads();
        for (int r = c + 1 + tid; r < n; r += blockDim.x) Pm[r * n + c] = 0.0;
        __syncthreads();
    }
    // back substitution, column-parallel over the RHS
    for (int col = tid; col < n; col += blockDim.x) {
        for (int r = n - 1; r >= 0; --r) {
            double v = Q[r * n + col];
            for (int k = r + 1; k < n; ++k) v -= Pm[r * n + k] * Q[k * n + col];
            Q[r * n + col] = v / Pm[r * n + r];
        }
    }
    __syncthreads();
    // Rm = Q.  Undo the scaling: Rm^(2^s) e_1 by squarings or repeated products.
    double* Rm = Q;
    const long long nmv = 1LL << s;
    if ((double)nmv <= (double)s * n) {
        double* x = A4;
        double* y = A6;
        for (int r = tid; r < n; r += blockDim.x) x[r] = (r == 0) ? 1.0 : 0.0;
        __syncthreads();
        for (long long it = 0; it < nmv; ++it) {
            for (int r = tid; r < n; r += blockDim.x) {
                double v = 0.0;
                for (int k = 0; k < n; ++k) v = fma(Rm[r * n + k], x[k], v);
                y[r] = v;
            }
            __syncthreads();
            for (int r = tid; r < n; r += blockDim.x) x[r] = y[r];
            __syncthreads();
        }
        for (int r = tid; r < n; r += blockDim.x) eo[r] = x[r];
    } else {
        double* cur = Rm;
        double* nxt = Um;
        for (int it = 0; it < s; ++it) {
            mat_mul(cur, cur, nxt, n);
            double* t = cur;
            cur = nxt;
            nxt = t;
        }
        for (int r = tid; r < n; r += blockDim.x) eo[r] = cur[r * n + 0];
    }
}

// ---------------------------------------------------------------- Faber coefficients
// a_j = (1/N) sum_k exp(dt psi(w_k)) w_k^-j on w_k = exp(2 pi i k / N),
// psi(w) = gamma (w + c0 + c1 / w); real part:
// exp(dt gamma (c0 + (1 + c1) cos th)) cos(dt gamma (1 - c1) sin th - j th).
__global__ void faber_coeff_kernel(double dt, double gamma, double c0, double c1, int m,
                                   int N, double* out) {
    __shared__ double red[8];
    const int j = blockIdx.x;
    if (j > m) return;
    double s = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double th = 2.0 * M_PI * (double)k / (double)N;
        double sn, cs;
        sincos(th, &sn, &cs);
        const double mag = exp(dt * gamma * (c0 + (1.0 + c1) * cs));
        s += mag * cos(dt * gamma * (1.0 - c1) * sn - (double)j * th);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
        out[j] = t / (double)N;
    }
}

// ---------------------------------------------------------------- launchers
void launch_set_clock(const ProblemDev* probs, int nprob, double t, double dt, cudaStream_t s) {
    set_clock_kernel<<<(nprob + 127) / 128, 128, 0, s>>>(probs, nprob, t, dt);
}
void launch_reset_cursor(const ProblemDev* probs, int nprob, cudaStream_t s) {
    reset_cursor_kernel<<<(nprob + 127) / 128, 128, 0, s>>>(probs, nprob);
}
void launch_prologue(const ProblemDev* probs, int nprob, int kind, int m, double gamma,
                     double c0, double c1, cudaStream_t s) {
    prologue_kernel<<<(nprob + 3) / 4, 128, 0, s>>>(probs, nprob, kind, m, gamma, c0, c1);
}
void launch_record(int precision, const ProblemDev* probs, int nprob, int vec, cudaStream_t s) {
    if (precision == 0) record_kernel<float><<<nprob, 128, 0, s>>>(probs, nprob, vec);
    else record_kernel<double><<<nprob, 128, 0, s>>>(probs, nprob, vec);
}
void launch_inject(int precision, void* adj, long long vec_elems, const void* values,
                   const int* rec_off, const int* nrec, int nshots, int max_rec, cudaStream_t s) {
    const int blocks = (nshots + 63) / 64;
    if (precision == 0)
        inject_kernel<float><<<blocks, 64, 0, s>>>((float*)adj, vec_elems, (const float*)values, rec_off,
                                                   nrec, nshots, max_rec);
    else
        inject_kernel<double><<<blocks, 64, 0, s>>>((double*)adj, vec_elems, (const double*)values,
                                                    rec_off, nrec, nshots, max_rec);
}

void launch_sum_shots(int precision, const void* in, void* out, long long n, int nshots,
                      cudaStream_t s) {
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (precision == 0) sum_shots_kernel<float><<<blocks, 256, 0, s>>>((const float*)in, (float*)out, n, nshots);
    else sum_shots_kernel<double><<<blocks, 256, 0, s>>>((const double*)in, (double*)out, n, nshots);
}

// Non-finite scan at the end of a step call: every block checks one PCHUNK chunk of its
// problem's state vector (the pads hold zeros) and the first block of each problem its
// Arnoldi flag; any NaN or infinity sets bit 1 (EWV error word: 1 = a pipeline wait timed
// out, 2 = a non-finite value) with one atomicOr per block that saw one.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
nonfinite_scan_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ pbase, int nprob,
                      int* err) {
    using V = typename Vec16<T>::type;
    constexpr int NV = Vec16<T>::N;
    const int pid = flat_problem(pbase, nprob, blockIdx.x);
    const ProblemDev* P = probs + pid;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nf = P->nfields;   // 4 (2D) or 6 (3D: w_z and psi added)
    const long long nelem = (long long)nf * P->field_stride;
    const int c = blockIdx.x - __ldg(pbase + pid);
    const long long e0 = (long long)c * PCHUNK;
    const long long e1 = e0 + PCHUNK < nelem ? e0 + PCHUNK : nelem;
    const V* S = reinterpret_cast<const V*>(vptr<T>(P, 0));
    bool bad = (c == 0 && tid == 0 && P->kry != nullptr && P->kry[KRY_NONFINITE] != 0.0);
    for (long long q = e0 / NV + tid; q < e1 / NV; q += NTHREADS) {
        const V v = S[q];
        bool b = !isfinite(v.x) || !isfinite(v.y);
        if constexpr (NV == 4) b = b || !isfinite(v.z) || !isfinite(v.w);
        bad = bad || b;
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(err, 2);
}

void launch_nonfinite_scan(int precision, int nchunks, const ProblemDev* probs, const int* pbase,
                           int nprob, int* err, cudaStream_t s) {
    if (nchunks <= 0) return;
    const dim3 block(TPX, TPY);
    if (precision == 0) nonfinite_scan_kernel<float><<<nchunks, block, 0, s>>>(probs, pbase, nprob, err);
    else nonfinite_scan_kernel<double><<<nchunks, block, 0, s>>>(probs, pbase, nprob, err);
}

void launch_point(int precision, int nblocks, const ProblemDev* probs, const int* tile_prob,
                  const PointArgs& pa, cudaStream_t s) {
    const dim3 block(TPX, TPY);
    if (precision == 0) point_kernel<float><<<nblocks, block, 0, s>>>(probs, tile_prob, pa);
    else point_kernel<double><<<nblocks, block, 0, s>>>(probs, tile_prob, pa);
}
void launch_point_flat(int precision, int nchunks, const ProblemDev* probs, const int* pbase,
                       int nprob, const PointArgs& pa, cudaStream_t s) {
    if (nchunks <= 0) return;
    const dim3 block(TPX, TPY);
    if (pa.mode == 8) {
        if (pa.nout + pa.final_out < 1 || pa.nout + pa.final_out > MAX_TAU || !pa.ecoef) return;
        if (precision == 0) combine_multi_kernel<float><<<nchunks, block, 0, s>>>(probs, pbase, nprob, pa);
        else combine_multi_kernel<double><<<nchunks, block, 0, s>>>(probs, pbase, nprob, pa);
        return;
    }
    if (precision == 0) point_flat_kernel<float><<<nchunks, block, 0, s>>>(probs, pbase, nprob, pa);
    else point_flat_kernel<double><<<nchunks, block, 0, s>>>(probs, pbase, nprob, pa);
}
static int launch_expm_taus(const ProblemDev* probs, int nprob, int mmax, cudaStream_t s, const ExpmTaus& et) {
    const size_t smem = (size_t)7 * mmax * mmax * sizeof(double);
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(expm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return -1;
    }
    expm_kernel<<<dim3(nprob, et.n), 256, smem, s>>>(probs, nprob, et);
    return 0;
}
int launch_expm(const ProblemDev* probs, int nprob, int mmax, cudaStream_t s, double hscale) {
    ExpmTaus et{};
    et.n = 1;
    et.tau[0] = hscale;
    et.out = nullptr;
    return launch_expm_taus(probs, nprob, mmax, s, et);
}
int launch_expm_multi(const ProblemDev* probs, int nprob, int mmax, cudaStream_t s, const double* taus, int ntau,
                      double* out) {
    if (ntau < 1 || ntau > MAX_TAU || !out) return -1;
    ExpmTaus et{};
    et.n = ntau;
    for (int q = 0; q < ntau; ++q) et.tau[q] = taus[q];
    et.out = out;
    return launch_expm_taus(probs, nprob, mmax, s, et);
}
void launch_faber_coeffs(double dt, double gamma, double c0, double c1, int m, double* out,
                         cudaStream_t s) {
    const int N = (4 * m > 64) ? 4 * m : 64;
    faber_coeff_kernel<<<m + 1, 256, 0, s>>>(dt, gamma, c0, c1, m, N, out);
}

}  // namespace ewv
