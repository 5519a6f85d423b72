// Exact discrete adjoint of the Krylov step: the reverse sweep through the Arnoldi process.
//
// The forward step (Sec. 3.2, Krylov listing, with the augmented matrix of Eq. matrix_ampli)
// maps U^n to U^{n+1} = beta [V_m expm(H_m) e_1]_U, with modified Gram-Schmidt Arnoldi on
// A = dt H~ from x = [U^n; eta e_p] (eta = |U^n|, the source column of H~ scaled by 1/eta).
// The basis and the Hessenberg matrix depend on U^n, so the step is nonlinear in U^n; this
// file runs the reverse mode of that map, operation by operation in the opposite order.
// api.cu recomputes the forward basis from the checkpoint, evaluates the small dense parts on
// the host in FP64 (the Frechet derivative of expm, read off the block exponential of
// [[H_m^T, E], [0, H_m^T]]) and sequences the passes below.
//
// The forward keeps the basis unnormalised: slot k holds q_k on the grid and its tail tau_k
// (p entries, FP64, in the Krylov scalar block), v_k = s_k (q_k, tau_k).  The reverse keeps
// the cotangents Vbar_k of v_k (grid vectors in the workspace, tails in the adjoint scalar
// block kbar), the cotangent wbar of the Arnoldi vector being orthogonalised and the
// forward vector w itself, rebuilt from the basis and H instead of stored:
//   w_before(k) = w_after(k) + h_{k,j} v_k.
// Column j of the reverse sweep, with Hbar from the output:
//   (normalisation, j < m_eff) hbar = Hbar_{j+1,j} - <Vbar_{j+1}, v_{j+1}> / h_{j+1,j},
//                              wbar = Vbar_{j+1} / h_{j+1,j} + hbar v_{j+1};  wbar = 0 for
//                              the last column;
//   (Gram-Schmidt, k = j .. k0) hbar = Hbar_{k,j} - <wbar, v_k>,
//                              Vbar_k += -h_{k,j} wbar + hbar w_before(k),
//                              wbar += hbar v_k
//                              (the forward skips the subtraction of k = m in the last
//                              column of a full-dimension step: there only the dot is reversed);
//   (matrix-vector product)    Vbar_j += dt H^T wbar_U (api.cu: transposed stencil pass),
//                              tail and source terms (launch_kadj_src), and
//                              grad += dt s_j wbar_v G(q_j) (api.cu: gradient pass).
// Every pass is one sweep over the padded vectors (pads are zero), fused with the next dot
// product where the order allows; a dot's partials are summed in a fixed order by the
// problem's last-arriving block, which runs the scalar step on one thread (deterministic).
#include "ewave_internal.cuh"
#include "krylov_finalize.cuh"

namespace ewv {

namespace {

template <typename T>
__device__ __forceinline__ T* kvec(const ProblemDev* P, int k) {
    return k == 0 ? (T*)P->state : (T*)P->work + (long long)(k - 1) * P->vec_stride;
}

__device__ __forceinline__ int kadj_problem(const int* __restrict__ base, int nprob, int b) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ const double* ktail(const double* kry, int k) {   // k = 1..MAX_M+1
    return kry + KRY_T + (k - 1) * MAX_P;
}
__device__ __forceinline__ double kh(const double* kry, int k, int j) {         // h_{k,j}
    return kry[KRY_H + (k - 1) * MAX_M + (j - 1)];
}

// True when the forward step at (column j, index k) took the dot product without the
// subtraction (the last column of a step that reached its full dimension m).
__device__ __forceinline__ bool dot_only(int j, int k, int m, int me) {
    return j == m && me == m && k == m;
}

// Scalar step after a dot product, one thread per problem.
__device__ void kadj_finalize(const ProblemDev* P, const KAdjArgs& ka, double tot) {
    const double* kry = P->kry;
    double* kb = P->kbar;
    const int p = P->p;
    const int me = (int)kry[KRY_MEFF];
    const int j = ka.j;
    switch (ka.fin) {
        case FK_STORE:
            kb[ka.slot] = tot;
            break;
        case FK_COLPREP: {
            double* wt = kb + KB_WT;
            double* ct = kb + KB_CT;
            const double* tn = ktail(kry, j + 1);
            if (j < me) {
                const double h = kh(kry, j + 1, j), s1 = kry[KRY_S + j + 1];
                const double* vt = kb + KB_VT + j * MAX_P;          // Vbar_{j+1}
                double full = tot;
                for (int q = 0; q < p; ++q) full += vt[q] * tn[q];
                const double hcol = kb[KB_HB + j * MAX_M + (j - 1)] - s1 * full / h;
                kb[KB_HCOL] = hcol;
                for (int q = 0; q < MAX_P; ++q) {
                    wt[q] = q < p ? vt[q] / h + hcol * s1 * tn[q] : 0.0;
                    ct[q] = q < p ? tn[q] : 0.0;
                }
            } else {
                kb[KB_HCOL] = 0.0;
                for (int q = 0; q < MAX_P; ++q) {
                    wt[q] = 0.0;
                    ct[q] = (j == me && q < p) ? tn[q] : 0.0;
                }
            }
            break;
        }
        case FK_GSPREP: {
            if (j > me) break;
            const int k = ka.fk;
            const double* tk = ktail(kry, k);
            const double sk = kry[KRY_S + k], hkj = kh(kry, k, j);
            double* wt = kb + KB_WT;
            double* ct = kb + KB_CT;
            double* vt = kb + KB_VT + (k - 1) * MAX_P;
            double full = tot;
            for (int q = 0; q < p; ++q) full += wt[q] * tk[q];
            const double hbar = kb[KB_HB + (k - 1) * MAX_M + (j - 1)] - sk * full;
            kb[KB_HBAR] = hbar;
            const bool only = dot_only(j, k, ka.m, me);
            for (int q = 0; q < p; ++q) {
                if (!only) {
                    ct[q] += hkj * sk * tk[q];
                    vt[q] += -hkj * wt[q] + hbar * ct[q];
                } else {
                    vt[q] += hbar * ct[q];
                }
                wt[q] += hbar * sk * tk[q];
            }
            break;
        }
        case FK_START: {
            const double beta = kry[KRY_BETA];
            const double* t1 = ktail(kry, 1);
            const double eta = t1[p - 1];
            const double* vt = kb + KB_VT;                           // Vbar_1
            double full = tot;
            for (int q = 0; q < p; ++q) full += vt[q] * t1[q];
            const double bbar = kb[KB_BBAR] - full / (beta * beta);
            const double xbar_last = vt[p - 1] / beta + bbar * eta / beta;
            const double ebar = kb[KB_EBAR] + xbar_last;
            // eta = |U| unless U = 0 (then eta = 1, beta = 1 and beta^2 - eta^2 = 0 exactly)
            const bool eta_const = !(beta * beta - eta * eta > 0.0);
            kb[KB_OA] = 1.0 / beta;
            kb[KB_OB] = bbar / beta + (eta_const ? 0.0 : ebar / eta);
            break;
        }
        default:
            break;
    }
}

template <typename T>
struct V16;
template <>
struct V16<float> {
    using type = float4;
    static constexpr int N = 4;
    __device__ static float4 fma(float a, float4 x, float4 y) {
        return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
    }
    __device__ static float4 scale(float a, float4 x) { return make_float4(a * x.x, a * x.y, a * x.z, a * x.w); }
    __device__ static double dot(float4 a, float4 b) {
        return (double)fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
    }
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct V16<double> {
    using type = double2;
    static constexpr int N = 2;
    __device__ static double2 fma(double a, double2 x, double2 y) {
        return make_double2(::fma(a, x.x, y.x), ::fma(a, x.y, y.y));
    }
    __device__ static double2 scale(double a, double2 x) { return make_double2(a * x.x, a * x.y); }
    __device__ static double dot(double2 a, double2 b) { return ::fma(a.y, b.y, a.x * b.x); }
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
};

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
kadj_flat_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ pbase, int nprob,
                 KAdjArgs ka) {
    using Ops = V16<T>;
    using V = typename Ops::type;
    constexpr int NV = Ops::N;
    __shared__ double red[NTHREADS / 32];
    __shared__ int s_last;
    const int pid = kadj_problem(pbase, nprob, blockIdx.x);
    const ProblemDev* P = probs + pid;
    const double* kry = P->kry;
    double* kb = P->kbar;
    const int me = (int)kry[KRY_MEFF];
    if (me <= 0 || kry[KRY_NONFINITE] != 0.0) return;          // nothing to reverse
    if (ka.mode == KA_GS && ka.j > me) return;                  // column beyond this problem
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const long long nelem = (long long)P->nfields * P->field_stride;
    const int c = blockIdx.x - __ldg(pbase + pid);
    const long long e0 = (long long)c * PCHUNK;
    const long long e1 = e0 + PCHUNK < nelem ? e0 + PCHUNK : nelem;
    const long long q0 = e0 / NV, q1 = e1 / NV;
    const int m = ka.m, j = ka.j;
    V* Wb = reinterpret_cast<V*>(kvec<T>(P, 2 * m + 3));
    V* Wc = reinterpret_cast<V*>(kvec<T>(P, 2 * m + 4));
    double acc = 0.0;
    switch (ka.mode) {
        case KA_DOT: {
            // the column-normalisation dot of the last column is not used: skip its vectors
            if (ka.fin == FK_COLPREP && j >= me) break;
            const V* A = reinterpret_cast<const V*>(kvec<T>(P, ka.a));
            const V* B = reinterpret_cast<const V*>(kvec<T>(P, ka.b));
            for (long long q = q0 + tid; q < q1; q += NTHREADS) acc += Ops::dot(A[q], B[q]);
            break;
        }
        case KA_SCALE: {
            const T cf = (T)kb[ka.slot];
            const V* A = reinterpret_cast<const V*>(kvec<T>(P, ka.a));
            V* B = reinterpret_cast<V*>(kvec<T>(P, ka.b));
            for (long long q = q0 + tid; q < q1; q += NTHREADS) B[q] = Ops::scale(cf, A[q]);
            break;
        }
        case KA_COLSET: {
            // wbar = Vbar_{j+1} / h_{j+1,j} + hbar v_{j+1}, v_{j+1} = s_{j+1} q_{j+1} (j < m_eff),
            // else 0; w = q_{j+1}; fused <wbar, q_j>
            const bool live = j < me;
            const T hinv = live ? (T)(1.0 / kh(kry, j + 1, j)) : T(0);
            const T cq = live ? (T)(kb[KB_HCOL] * kry[KRY_S + j + 1]) : T(0);
            const V* Qn = reinterpret_cast<const V*>(kvec<T>(P, j + 1));
            const V* Vb = reinterpret_cast<const V*>(kvec<T>(P, m + 2 + j));
            const V* Qd = ka.dot >= 0 && j <= me ? reinterpret_cast<const V*>(kvec<T>(P, ka.dot)) : nullptr;
            // every operand is loaded before the stores (one memory round trip per element)
            for (long long q = q0 + tid; q < q1; q += NTHREADS) {
                const V qn = Qn[q];
                const V vbq = Vb[q];
                const V qd = Qd ? Qd[q] : Ops::zero();
                const V wb = live ? Ops::fma(cq, qn, Ops::scale(hinv, vbq)) : Ops::zero();
                Wb[q] = wb;
                Wc[q] = qn;
                if (Qd) acc += Ops::dot(wb, qd);
            }
            break;
        }
        case KA_GS: {
            const int k = ka.k;
            const T hbar = (T)kb[KB_HBAR];
            const T hs = (T)(kh(kry, k, j) * kry[KRY_S + k]);   // h_{k,j} s_k
            const T hkj = (T)kh(kry, k, j);
            const T hbs = (T)(kb[KB_HBAR] * kry[KRY_S + k]);    // hbar s_k
            const bool only = dot_only(j, k, m, me);
            const V* Qk = reinterpret_cast<const V*>(kvec<T>(P, k));
            V* Vb = reinterpret_cast<V*>(kvec<T>(P, m + 1 + k));
            const V* Qd = ka.dot >= 0 ? reinterpret_cast<const V*>(kvec<T>(P, ka.dot)) : nullptr;
            for (long long q = q0 + tid; q < q1; q += NTHREADS) {
                const V qk = Qk[q];
                const V wb = Wb[q];
                V wc = Wc[q];
                V vb = Vb[q];
                const V qd = Qd ? Qd[q] : Ops::zero();   // before the stores, as above
                if (!only) {
                    wc = Ops::fma(hs, qk, wc);                 // w_before(k)
                    Wc[q] = wc;
                    vb = Ops::fma(-hkj, wb, vb);
                }
                Vb[q] = Ops::fma(hbar, wc, vb);
                const V wn = Ops::fma(hbs, qk, wb);
                Wb[q] = wn;
                if (Qd) acc += Ops::dot(wn, qd);
            }
            break;
        }
        case KA_OUT: {
            const T a = (T)kb[KB_OA], b = (T)kb[KB_OB];
            const V* V1 = reinterpret_cast<const V*>(kvec<T>(P, m + 2));
            const V* Q1 = reinterpret_cast<const V*>(kvec<T>(P, 1));
            V* L = reinterpret_cast<V*>(kvec<T>(P, 0));
            for (long long q = q0 + tid; q < q1; q += NTHREADS) L[q] = Ops::fma(b, Q1[q], Ops::scale(a, V1[q]));
            break;
        }
        default:
            break;
    }
    if (ka.fin == FK_NONE) return;
    // fixed-order sum of the problem's partials by its last-arriving block
    const double bsum = block_sum_fixed(acc, red);
    if (tid == 0) {
        ka.partials[blockIdx.x] = bsum;
        __threadfence();
        const unsigned int prev = atomicAdd(ka.counters + pid, 1u);
        s_last = (prev == (unsigned int)(P->pchunks - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int base = __ldg(pbase + pid);
    double v = 0.0;
    for (int t = tid; t < P->pchunks; t += NTHREADS) v += __ldcg(ka.partials + base + t);
    const double tot = block_sum_fixed(v, red);
    if (tid == 0) {
        kadj_finalize(P, ka, tot);
        ka.counters[pid] = 0u;
        __threadfence();
    }
}

// Tail and source terms of the reverse matrix-vector product w = A v_j (one thread per
// problem): Vbar_j tail += J^T wbar_tail + dt (W / eta) wbar_v[src], and
// eta_bar -= dt wbar_v[src] (W_raw . y_j) / eta^2 with y_j = s_j tau_j, W_raw = eta W.
template <typename T>
__global__ void kadj_src_kernel(const ProblemDev* probs, int nprob, int j, int m, double dt) {
    const int pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= nprob) return;
    const ProblemDev* P = probs + pid;
    const double* kry = P->kry;
    double* kb = P->kbar;
    const int me = (int)kry[KRY_MEFF];
    if (me <= 0 || kry[KRY_NONFINITE] != 0.0 || j > me) return;
    const int p = P->p;
    const double* wt = kb + KB_WT;
    double* vt = kb + KB_VT + (j - 1) * MAX_P;
    for (int q = p - 1; q >= 1; --q) vt[q] += wt[q - 1];
    if (P->has_src) {
        const T* wb = kvec<T>(P, 2 * m + 3);
        const long long o = P->field_stride + (long long)P->src_j * P->pitch + P->src_i;
        const double ws = (double)wb[o];
        const double* W = kry + KRY_W;
        const double* tj = ktail(kry, j);
        const double eta = ktail(kry, 1)[p - 1];
        double wy = 0.0;
        for (int q = 0; q < p; ++q) {
            vt[q] += dt * W[q] * ws;
            wy += W[q] * tj[q];
        }
        kb[KB_EBAR] -= dt * ws * kry[KRY_S + j] * wy / eta;
    }
}

}  // namespace

void launch_kadj_flat(int precision, int nchunks, const ProblemDev* probs, const int* pbase,
                      int nprob, const KAdjArgs& ka, cudaStream_t s) {
    if (nchunks <= 0) return;
    const dim3 block(TPX, TPY);
    if (precision == 0) kadj_flat_kernel<float><<<nchunks, block, 0, s>>>(probs, pbase, nprob, ka);
    else kadj_flat_kernel<double><<<nchunks, block, 0, s>>>(probs, pbase, nprob, ka);
}

void launch_kadj_src(const ProblemDev* probs, int nprob, int precision, int j, int m, double dt,
                     cudaStream_t s) {
    const int blocks = (nprob + 63) / 64;
    if (precision == 0) kadj_src_kernel<float><<<blocks, 64, 0, s>>>(probs, nprob, j, m, dt);
    else kadj_src_kernel<double><<<blocks, 64, 0, s>>>(probs, nprob, j, m, dt);
}

}  // namespace ewv
