// Fused stencil kernels: one HBM-streaming pass applies the operator H of Eq. (1) (or its
// transpose) to a state vector and folds in the integrator's recurrence / accumulation,
// so that every Faber degree, HORK/RK stage and Krylov matrix-vector product is one pass.
//
// Operator (Eq. 1, Sec. 2): for U = (u, v, w_x, w_y)
//   (HU)_u   = v
//   (HU)_v   = -bx by u + c^2 (u_xx + u_yy) - (bx + by) v + c^2 (d_x w_x + d_y w_y)
//   (HU)_w_x = (by - bx) d_x u - bx w_x         at (i+1/2, j)
//   (HU)_w_y = (bx - by) d_y u - by w_y         at (i, j+1/2)
// with Sec. 2.1's staggered 8th-order first derivative (Eq. spatial_8th_1) and centred
// second derivative (Eq. spatial_8th_2, "+" between the symmetric pairs), 4th-order
// textbook tables for fd_order 4, zero extension beyond the grid, and -- with a free
// surface -- Appendix A's one-sided rows for u_yy (rows 0..3) and u_y (half rows 0..2) and
// Fornberg rows (Sec. 2.2) for d_y w_y (rows 0..3).  y is the paper's upward axis, the row
// index j grows downward: d_y u at half row j+1/2 = sum_k s_k (u_{j-k} - u_{j+1+k}) / dx.
// The damping beta = beta0 (1 - d/delta)^2 (Sec. 2) is evaluated in registers from the
// node / half-node distance to the first ghost line.
//
// Layout: per block a BX x BY tile of outputs.  u is staged in shared memory with an
// R-wide halo on all sides, w_x with an x halo, w_y with a y halo (zero outside the grid =
// the zero extension); v, c^2 and the integrator's pointwise operands are read straight
// from global memory (coalesced) and prefetched before the staging barrier.
//
// Epilogue (StageArgs), per field f at every output point:
//   K   = cx X + ch xs (H X + sigma e_src)          (xs: per-problem scale, Krylov)
//   Y   = cu U + ck K                               -> y_out
//   ACC = ca A + cau U + cak K + cay Y + cax X      -> acc_out
// and optionally a partial dot product <Y, D> (Krylov), finalised by the last block.
#include <cuda_bf16.h>

#include <type_traits>

#include "ewave_internal.cuh"
#include "krylov_finalize.cuh"

namespace ewv {

// Free-surface tables: Appendix A rows (library's own copy of the printed rationals) and
// the Fornberg d_y w_y rows computed on the host at model creation.
__constant__ double g_fs_d[4 * 9 + 3 * 8 + 4 * 8];
__constant__ float g_fs_f[4 * 9 + 3 * 8 + 4 * 8];
constexpr int FS_UYY_OFF = 0, FS_UY_OFF = 36, FS_DWY_OFF = 60;

int upload_stencil_tables(int /*order*/, const double* fs_uyy, const double* fs_uy,
                          const double* fs_dwy) {
    double d[92];
    float f[92];
    for (int i = 0; i < 36; ++i) d[FS_UYY_OFF + i] = fs_uyy[i];
    for (int i = 0; i < 24; ++i) d[FS_UY_OFF + i] = fs_uy[i];
    for (int i = 0; i < 32; ++i) d[FS_DWY_OFF + i] = fs_dwy[i];
    for (int i = 0; i < 92; ++i) f[i] = (float)d[i];
    if (cudaMemcpyToSymbol(g_fs_d, d, sizeof(d)) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(g_fs_f, f, sizeof(f)) != cudaSuccess) return -1;
    return 0;
}

template <typename T>
__device__ __forceinline__ T fs_coef(int off) {
    if constexpr (std::is_same<T, float>::value) return g_fs_f[off];
    else return g_fs_d[off];
}

// Interior tables (Eqs. spatial_8th_1/2 for R = 4; classical 4th-order tables for R = 2).
template <typename T, int R>
__device__ __forceinline__ T STAG(int k) {
    if constexpr (R == 4) {
        return k == 0 ? T(1225.0 / 1024.0) : k == 1 ? T(-245.0 / 3072.0)
             : k == 2 ? T(49.0 / 5120.0) : T(-5.0 / 7168.0);
    } else {
        return k == 0 ? T(9.0 / 8.0) : T(-1.0 / 24.0);
    }
}
template <typename T, int R>
__device__ __forceinline__ T CENT(int k) {
    if constexpr (R == 4) {
        return k == 0 ? T(-205.0 / 72.0) : k == 1 ? T(8.0 / 5.0) : k == 2 ? T(-1.0 / 5.0)
             : k == 3 ? T(8.0 / 315.0) : T(-1.0 / 560.0);
    } else {
        return k == 0 ? T(-5.0 / 2.0) : k == 1 ? T(4.0 / 3.0) : T(-1.0 / 12.0);
    }
}

// beta0 (1 - d/delta)^2 for d <= delta, d in grid units.
template <typename T>
__device__ __forceinline__ T damp(T beta0, T inv_pml, T d, int pml) {
    if (pml <= 0) return T(0);
    const T r = T(1) - d * inv_pml;
    return (d <= T(pml)) ? beta0 * r * r : T(0);
}

// Round to the nearest bfloat16 (ties to even) and widen back: the value that a bfloat16
// store followed by a load would return.
template <typename T>
__device__ __forceinline__ T bf16_round(T v) {
    return (T)__bfloat162float(__float2bfloat16_rn((float)v));
}

template <typename T>
__device__ __forceinline__ T* vec_ptr(const ProblemDev* P, int k) {
    return k == 0 ? (T*)P->state : (T*)P->work + (long long)(k - 1) * P->vec_stride;
}

// --------------------------------------------------------------------------------------
// Stage kernel
// --------------------------------------------------------------------------------------
template <typename T, int R, bool TRANS>
__global__ void __launch_bounds__(NTHREADS)
stage_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tile_prob,
             StageArgs a) {
    constexpr int SW = BX + 2 * R;    // staged width with x halo
    constexpr int SH = BY + 2 * R;    // staged height with y halo
    __shared__ T su[SH][SW];
    __shared__ T swx[BY][SW];
    __shared__ T swy[SH][BX];
    __shared__ double red[NTHREADS / 32];
    __shared__ int s_last;

    const int pid = tile_prob[blockIdx.x];
    const ProblemDev* P = probs + pid;
    if (a.fin_mode != FIN_NONE && P->kry[KRY_ACTIVE] == 0.0) return;   // Arnoldi stopped

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = P->nx, ny = P->ny, pitch = P->pitch, pml = P->pml;
    const bool fs = P->fs != 0;
    const int lt = blockIdx.x - P->tile_base;
    const int x0 = (lt % P->tiles_x) * BX;
    const int y0 = (lt / P->tiles_x) * BY;
    const long long fstr = P->field_stride;
    const T beta0 = (T)P->beta0, inv_pml = (T)P->inv_pml;
    const T idx1 = (T)P->inv_dx, idx2 = (T)P->inv_dx2;

    const T* X = vec_ptr<T>(P, a.x);
    const T* C2 = (const T*)P->c2;

    // ---- prefetch pointwise operands (registers) ---------------------------------------
    T pv[VY][VX], pc2[VY][VX];
    T pU[4][VY][VX], pA[4][VY][VX];
    const T* U = a.u >= 0 ? vec_ptr<T>(P, a.u) : nullptr;
    const T* A = a.a >= 0 ? vec_ptr<T>(P, a.a) : nullptr;
#pragma unroll
    for (int b = 0; b < VY; ++b) {
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int i = x0 + tx + c * TPX, j = y0 + ty + b * TPY;
            const bool in = (i < nx) && (j < ny);
            const long long o = (long long)j * pitch + i;
            pv[b][c] = in ? X[fstr + o] : T(0);
            pc2[b][c] = in ? C2[o] : T(0);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                pU[f][b][c] = (in && U) ? U[f * fstr + o] : T(0);
                pA[f][b][c] = (in && A) ? A[f * fstr + o] : T(0);
            }
        }
    }

    // ---- stage halo tiles ----------------------------------------------------------------
    // Row-wise: thread (tx, ty) fills columns tx, tx + TPX, ... of rows ty, ty + TPY, ...; the
    // row's bounds test and (in the transpose) its damping factor are taken once per row.
    if constexpr (!TRANS) {
        const T* Xu = X;
        const T* Xwx = X + 2 * fstr;
        const T* Xwy = X + 3 * fstr;
        for (int r = ty; r < SH; r += TPY) {
            const int gy = y0 - R + r;
            const bool rok = gy >= 0 && gy < ny;
            const T* row = Xu + (long long)(rok ? gy : 0) * pitch;
            for (int c = tx; c < SW; c += TPX) {
                const int gx = x0 - R + c;
                su[r][c] = (rok && gx >= 0 && gx < nx) ? row[gx] : T(0);
            }
        }
        for (int r = ty; r < BY; r += TPY) {
            const int gy = y0 + r;
            const bool rok = gy < ny;
            const T* row = Xwx + (long long)(rok ? gy : 0) * pitch;
            for (int c = tx; c < SW; c += TPX) {
                const int gx = x0 - R + c;
                swx[r][c] = (rok && gx >= 0 && gx < nx - 1) ? row[gx] : T(0);
            }
        }
        for (int r = ty; r < SH; r += TPY) {
            const int gy = y0 - R + r;
            const bool rok = gy >= 0 && gy < ny - 1;
            const T* row = Xwy + (long long)(rok ? gy : 0) * pitch;
            for (int c = tx; c < BX; c += TPX) {
                const int gx = x0 + c;
                swy[r][c] = (rok && gx < nx) ? row[gx] : T(0);
            }
        }
    } else {
        // Transpose: stage z_v = c^2 y_v (2D halo), z_x = g_x y_wx (x halo) and
        // z_y = g_y y_wy (y halo), g_x = by(j) - bx(i+1/2), g_y = bx(i) - by(j+1/2).
        const T* Xv = X + fstr;
        const T* Xwx = X + 2 * fstr;
        const T* Xwy = X + 3 * fstr;
        for (int r = ty; r < SH; r += TPY) {
            const int gy = y0 - R + r;
            const bool rok = gy >= 0 && gy < ny;
            const long long ro = (long long)(rok ? gy : 0) * pitch;
            for (int c = tx; c < SW; c += TPX) {
                const int gx = x0 - R + c;
                su[r][c] = (rok && gx >= 0 && gx < nx) ? C2[ro + gx] * Xv[ro + gx] : T(0);
            }
        }
        for (int r = ty; r < BY; r += TPY) {
            const int gy = y0 + r;
            const bool rok = gy < ny;
            const T* row = Xwx + (long long)(rok ? gy : 0) * pitch;
            const T byn = rok ? damp<T>(beta0, inv_pml, fs ? T(ny - gy) : T(min(gy + 1, ny - gy)), pml) : T(0);
            for (int c = tx; c < SW; c += TPX) {
                const int gx = x0 - R + c;
                T val = T(0);
                if (rok && gx >= 0 && gx < nx - 1) {
                    const T dxh = min(T(gx) + T(1.5), T(nx - gx) - T(0.5));
                    val = (byn - damp<T>(beta0, inv_pml, dxh, pml)) * row[gx];
                }
                swx[r][c] = val;
            }
        }
        for (int r = ty; r < SH; r += TPY) {
            const int gy = y0 - R + r;
            const bool rok = gy >= 0 && gy < ny - 1;
            const T* row = Xwy + (long long)(rok ? gy : 0) * pitch;
            const T byh = rok ? damp<T>(beta0, inv_pml,
                                        fs ? (T(ny - gy) - T(0.5)) : min(T(gy) + T(1.5), T(ny - gy) - T(0.5)), pml)
                              : T(0);
            for (int c = tx; c < BX; c += TPX) {
                const int gx = x0 + c;
                T val = T(0);
                if (rok && gx < nx) val = (damp<T>(beta0, inv_pml, T(min(gx + 1, nx - gx)), pml) - byh) * row[gx];
                swy[r][c] = val;
            }
        }
    }
    __syncthreads();

    const T cx = (T)a.cx, ch = (T)a.ch, cu = (T)a.cu, ck = (T)a.ck, ca = (T)a.ca;
    const T cau = (T)a.cau, cak = (T)a.cak, cay = (T)a.cay, cax = (T)a.cax;
    const T xs = a.x_scale_slot >= 0 ? (T)P->kry[a.x_scale_slot] : T(1);
    const T sig = (a.src_slot >= 0 && P->has_src) ? (T)P->sigma[a.src_slot] : T(0);
    T* Y = a.y_out >= 0 ? vec_ptr<T>(P, a.y_out) : nullptr;
    T* ACC = a.acc_out >= 0 ? vec_ptr<T>(P, a.acc_out) : nullptr;
    const T* D = a.d >= 0 ? vec_ptr<T>(P, a.d) : nullptr;
    float dotf = 0.f;
    double dotd = 0.0;

#pragma unroll
    for (int b = 0; b < VY; ++b) {
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int lx = tx + c * TPX, ly = ty + b * TPY;
            const int i = x0 + lx, j = y0 + ly;
            if (i >= nx || j >= ny) continue;
            const long long o = (long long)j * pitch + i;
            // damping at this node and its two half points
            const T bxn = damp<T>(beta0, inv_pml, T(min(i + 1, nx - i)), pml);
            const T byn = damp<T>(beta0, inv_pml, fs ? T(ny - j) : T(min(j + 1, ny - j)), pml);
            const T bxh = damp<T>(beta0, inv_pml, min(T(i) + T(1.5), T(nx - i) - T(0.5)), pml);
            const T byh = damp<T>(beta0, inv_pml,
                                  fs ? (T(ny - j) - T(0.5)) : min(T(j) + T(1.5), T(ny - j) - T(0.5)),
                                  pml);
            const T c2 = pc2[b][c];
            T xu, xv, xwx, xwy, hu, hv, hwx, hwy;
            if constexpr (!TRANS) {
                xu = su[ly + R][lx + R];
                xv = pv[b][c];
                xwx = swx[ly][lx + R];
                xwy = swy[ly + R][lx];
                // u_xx
                T uxx = CENT<T, R>(0) * xu;
#pragma unroll
                for (int k = 1; k <= R; ++k)
                    uxx += CENT<T, R>(k) * (su[ly + R][lx + R + k] + su[ly + R][lx + R - k]);
                // u_yy
                T uyy;
                if (fs && j < 4) {
                    uyy = T(0);
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        uyy += fs_coef<T>(FS_UYY_OFF + j * 9 + q) * su[q - y0 + R][lx + R];
                } else {
                    uyy = CENT<T, R>(0) * xu;
#pragma unroll
                    for (int k = 1; k <= R; ++k)
                        uyy += CENT<T, R>(k) * (su[ly + R + k][lx + R] + su[ly + R - k][lx + R]);
                }
                // d_x w_x at the node: w_x[i+k] - w_x[i-1-k]
                T dwx = T(0);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    dwx += STAG<T, R>(k) * (swx[ly][lx + R + k] - swx[ly][lx + R - 1 - k]);
                // d_y w_y at the node (upward y): w_y[j-1-k] - w_y[j+k]
                T dwy = T(0);
                if (fs && j < 4) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        dwy += fs_coef<T>(FS_DWY_OFF + j * 8 + q) * swy[q - y0 + R][lx];
                } else {
#pragma unroll
                    for (int k = 0; k < R; ++k)
                        dwy += STAG<T, R>(k) * (swy[ly + R - 1 - k][lx] - swy[ly + R + k][lx]);
                }
                // d_x u at (i+1/2, j)
                T dux = T(0);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    dux += STAG<T, R>(k) * (su[ly + R][lx + R + 1 + k] - su[ly + R][lx + R - k]);
                // d_y u at (i, j+1/2)
                T duy = T(0);
                if (fs && j < 3) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        duy += fs_coef<T>(FS_UY_OFF + j * 8 + q) * su[q - y0 + R][lx + R];
                } else {
#pragma unroll
                    for (int k = 0; k < R; ++k)
                        duy += STAG<T, R>(k) * (su[ly + R - k][lx + R] - su[ly + R + 1 + k][lx + R]);
                }
                if (a.grad) {
                    // FWI gradient w.r.t. m = c^2: d(H X)_v / dm = L X_u + D X_w
                    T* G = (T*)a.grad + (long long)P->shot * fstr;
                    const T* Q = vec_ptr<T>(P, a.gq);
                    const T gval = (uxx + uyy) * idx2 + (dwx + dwy) * idx1;
                    G[o] += (T)a.gscale * xs * Q[fstr + o] * gval;   // xs: per-problem scale
                    continue;
                }
                hu = xv;
                hv = -bxn * byn * xu + c2 * ((uxx + uyy) * idx2 + (dwx + dwy) * idx1)
                     - (bxn + byn) * xv;
                hwx = (i < nx - 1) ? (byn - bxh) * dux * idx1 - bxh * xwx : T(0);
                hwy = (j < ny - 1) ? (bxn - byh) * duy * idx1 - byh * xwy : T(0);
                if (i == P->src_i && j == P->src_j) hv += sig;
            } else {
                // H^T y.  Pointwise inputs: y_u (not staged), y_v = pv, y_wx, y_wy from the
                // unscaled vector; staged: zv = c^2 y_v, zx = g_x y_wx, zy = g_y y_wy.
                const T* Xg = X;
                xu = Xg[o];
                xv = pv[b][c];
                xwx = (i < nx - 1) ? Xg[2 * fstr + o] : T(0);
                xwy = (j < ny - 1) ? Xg[3 * fstr + o] : T(0);
                // (Lxx^T zv)(i) = Lxx zv (symmetric)
                T lxx = CENT<T, R>(0) * su[ly + R][lx + R];
#pragma unroll
                for (int k = 1; k <= R; ++k)
                    lxx += CENT<T, R>(k) * (su[ly + R][lx + R + k] + su[ly + R][lx + R - k]);
                // (Lyy^T zv)(j): interior rows r >= rfs contribute CENT(|r-j|), free-surface
                // rows r < 4 contribute FS_UYY[r][j] for j <= 8.
                T lyy = T(0);
                const int rfs = fs ? 4 : 0;
#pragma unroll
                for (int k = -R; k <= R; ++k) {
                    const int r = j + k;
                    if (r >= rfs && r < ny) lyy += CENT<T, R>(k < 0 ? -k : k) * su[ly + R + k][lx + R];
                }
                if (fs && j <= 8) {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r < ny) lyy += fs_coef<T>(FS_UYY_OFF + r * 9 + j) * su[r - y0 + R][lx + R];
                }
                // (Dxh^T zx)(i) = sum_k s_k (zx[i-1-k] - zx[i+k])
                T gxt = T(0);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    gxt += STAG<T, R>(k) * (swx[ly][lx + R - 1 - k] - swx[ly][lx + R + k]);
                // (Dyh^T zy)(j): interior half rows h >= hfs: d_y u at h uses
                // s_k (u[h-k] - u[h+1+k]); free-surface half rows h < 3 use FS_UY[h][j].
                T gyt = T(0);
                const int hfs = fs ? 3 : 0;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int h1 = j + k;        // u[j] = u[h1 - k] with + sign
                    const int h2 = j - 1 - k;    // u[j] = u[h2 + 1 + k] with - sign
                    if (h1 >= hfs && h1 < ny - 1) gyt += STAG<T, R>(k) * swy[ly + R + k][lx];
                    if (h2 >= hfs && h2 >= 0) gyt -= STAG<T, R>(k) * swy[ly + R - 1 - k][lx];
                }
                if (fs && j <= 7) {
#pragma unroll
                    for (int h = 0; h < 3; ++h)
                        if (h < ny - 1) gyt += fs_coef<T>(FS_UY_OFF + h * 8 + j) * swy[h - y0 + R][lx];
                }
                // (Dxn^T zv)(i+1/2) = sum_k s_k (zv[i-k] - zv[i+1+k])
                T dxt = T(0);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    dxt += STAG<T, R>(k) * (su[ly + R][lx + R - k] - su[ly + R][lx + R + 1 + k]);
                // (Dyn^T zv)(j+1/2): interior rows r >= rfs: d_y w_y at r uses
                // s_k (w[r-1-k] - w[r+k]); free-surface rows r < 4 use FS_DWY[r][j].
                T dyt = T(0);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int r1 = j + 1 + k;    // w[j] = w[r1 - 1 - k], + sign
                    const int r2 = j - k;        // w[j] = w[r2 + k], - sign
                    if (r1 >= rfs && r1 < ny) dyt += STAG<T, R>(k) * su[ly + R + 1 + k][lx + R];
                    if (r2 >= rfs && r2 >= 0) dyt -= STAG<T, R>(k) * su[ly + R - k][lx + R];
                }
                if (fs && j <= 7) {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r < ny) dyt += fs_coef<T>(FS_DWY_OFF + r * 8 + j) * su[r - y0 + R][lx + R];
                }
                hu = -bxn * byn * xv + (lxx + lyy) * idx2 + (gxt + gyt) * idx1;
                hv = xu - (bxn + byn) * xv;
                hwx = (i < nx - 1) ? dxt * idx1 - bxh * xwx : T(0);
                hwy = (j < ny - 1) ? dyt * idx1 - byh * xwy : T(0);
            }
            // ---- epilogue ------------------------------------------------------------
            const T xf[4] = {xu, xv, xwx, xwy};
            const T hf[4] = {hu, hv, hwx, hwy};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const bool pad = (f == 2 && i >= nx - 1) || (f == 3 && j >= ny - 1);
                const T kf = cx * xs * xf[f] + ch * xs * hf[f];
                T yf = pad ? T(0) : (cu * pU[f][b][c] + ck * kf);
                if (a.store_bf16) yf = bf16_round(yf);     // storage-precision experiment
                if (Y) Y[f * fstr + o] = yf;
                if (ACC) {
                    T af = ca * pA[f][b][c] + cau * pU[f][b][c] + cak * kf + cay * yf
                           + cax * xs * xf[f];
                    if (a.store_bf16) af = bf16_round(af);
                    ACC[f * fstr + o] = pad ? T(0) : af;
                }
                if (D && !pad) {
                    const T dv = D[f * fstr + o];
                    if constexpr (std::is_same<T, float>::value) dotf = fmaf(yf, dv, dotf);
                    else dotd = fma(yf, dv, dotd);
                }
            }
        }
    }
    if (a.fin_mode != FIN_NONE) {
        const double mine = (double)dotf + dotd;
        const double bsum = block_sum_fixed(mine, red);
        partial_and_finalize(P, pid, a, bsum, red, &s_last);
    }
}

// --------------------------------------------------------------------------------------
// Leap-frog kernel (Sec. 3.1).  Vectors `cur` (u^n, w^n) and `prev` (u^{n-1}, w^{n-1}) use
// fields 0 (u), 2 (w_x), 3 (w_y); level n+1 overwrites `prev`.  Variant 2 (difference form)
// reads d^n = u^n - u^{n-1} from field 1 of `prev` instead of u^{n-1} and writes d^{n+1} to
// field 1 of `cur` (read by no other thread of the step), u^{n+1} = u^n + d^{n+1}.
// --------------------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(NTHREADS)
leapfrog_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tile_prob,
                int cur, int prev, int variant, double dt_d) {
    constexpr int SW = BX + 2 * R;
    constexpr int SH = BY + 2 * R;
    __shared__ T su[SH][SW];
    __shared__ T swx[BY][SW];
    __shared__ T swy[SH][BX];
    const int pid = tile_prob[blockIdx.x];
    const ProblemDev* P = probs + pid;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = P->nx, ny = P->ny, pitch = P->pitch, pml = P->pml;
    const bool fs = P->fs != 0;
    const int lt = blockIdx.x - P->tile_base;
    const int x0 = (lt % P->tiles_x) * BX, y0 = (lt / P->tiles_x) * BY;
    const long long fstr = P->field_stride;
    const T beta0 = (T)P->beta0, inv_pml = (T)P->inv_pml;
    const T idx1 = (T)P->inv_dx, idx2 = (T)P->inv_dx2;
    const T dt = (T)dt_d;
    T* Cn = vec_ptr<T>(P, cur);
    T* Pn = vec_ptr<T>(P, prev);
    const T* C2 = (const T*)P->c2;
    T pum[VY][VX], pwxm[VY][VX], pwym[VY][VX], pc2[VY][VX];
#pragma unroll
    for (int b = 0; b < VY; ++b)
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int i = x0 + tx + c * TPX, j = y0 + ty + b * TPY;
            const bool in = (i < nx) && (j < ny);
            const long long o = (long long)j * pitch + i;
            pum[b][c] = in ? Pn[(variant == 2 ? fstr : 0) + o] : T(0);
            pwxm[b][c] = in ? Pn[2 * fstr + o] : T(0);
            pwym[b][c] = in ? Pn[3 * fstr + o] : T(0);
            pc2[b][c] = in ? C2[o] : T(0);
        }
    for (int r = ty; r < SH; r += TPY) {
        const int gy = y0 - R + r;
        const bool rok = gy >= 0 && gy < ny;
        const T* row = Cn + (long long)(rok ? gy : 0) * pitch;
        for (int c = tx; c < SW; c += TPX) {
            const int gx = x0 - R + c;
            su[r][c] = (rok && gx >= 0 && gx < nx) ? row[gx] : T(0);
        }
    }
    for (int r = ty; r < BY; r += TPY) {
        const int gy = y0 + r;
        const bool rok = gy < ny;
        const T* row = Cn + 2 * fstr + (long long)(rok ? gy : 0) * pitch;
        for (int c = tx; c < SW; c += TPX) {
            const int gx = x0 - R + c;
            swx[r][c] = (rok && gx >= 0 && gx < nx - 1) ? row[gx] : T(0);
        }
    }
    for (int r = ty; r < SH; r += TPY) {
        const int gy = y0 - R + r;
        const bool rok = gy >= 0 && gy < ny - 1;
        const T* row = Cn + 3 * fstr + (long long)(rok ? gy : 0) * pitch;
        for (int c = tx; c < BX; c += TPX) {
            const int gx = x0 + c;
            swy[r][c] = (rok && gx < nx) ? row[gx] : T(0);
        }
    }
    __syncthreads();
    const T sig = P->has_src ? (T)P->sigma[0] : T(0);
#pragma unroll
    for (int b = 0; b < VY; ++b)
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int lx = tx + c * TPX, ly = ty + b * TPY;
            const int i = x0 + lx, j = y0 + ly;
            if (i >= nx || j >= ny) continue;
            const long long o = (long long)j * pitch + i;
            const T bxn = damp<T>(beta0, inv_pml, T(min(i + 1, nx - i)), pml);
            const T byn = damp<T>(beta0, inv_pml, fs ? T(ny - j) : T(min(j + 1, ny - j)), pml);
            const T bxh = damp<T>(beta0, inv_pml, min(T(i) + T(1.5), T(nx - i) - T(0.5)), pml);
            const T byh = damp<T>(beta0, inv_pml,
                                  fs ? (T(ny - j) - T(0.5)) : min(T(j) + T(1.5), T(ny - j) - T(0.5)),
                                  pml);
            const T u = su[ly + R][lx + R];
            T uxx = CENT<T, R>(0) * u;
#pragma unroll
            for (int k = 1; k <= R; ++k)
                uxx += CENT<T, R>(k) * (su[ly + R][lx + R + k] + su[ly + R][lx + R - k]);
            T uyy;
            if (fs && j < 4) {
                uyy = T(0);
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    uyy += fs_coef<T>(FS_UYY_OFF + j * 9 + q) * su[q - y0 + R][lx + R];
            } else {
                uyy = CENT<T, R>(0) * u;
#pragma unroll
                for (int k = 1; k <= R; ++k)
                    uyy += CENT<T, R>(k) * (su[ly + R + k][lx + R] + su[ly + R - k][lx + R]);
            }
            T dwx = T(0);
#pragma unroll
            for (int k = 0; k < R; ++k)
                dwx += STAG<T, R>(k) * (swx[ly][lx + R + k] - swx[ly][lx + R - 1 - k]);
            T dwy = T(0);
            if (fs && j < 4) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dwy += fs_coef<T>(FS_DWY_OFF + j * 8 + q) * swy[q - y0 + R][lx];
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k)
                    dwy += STAG<T, R>(k) * (swy[ly + R - 1 - k][lx] - swy[ly + R + k][lx]);
            }
            T dux = T(0);
#pragma unroll
            for (int k = 0; k < R; ++k)
                dux += STAG<T, R>(k) * (su[ly + R][lx + R + 1 + k] - su[ly + R][lx + R - k]);
            T duy = T(0);
            if (fs && j < 3) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    duy += fs_coef<T>(FS_UY_OFF + j * 8 + q) * su[q - y0 + R][lx + R];
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k)
                    duy += STAG<T, R>(k) * (su[ly + R - k][lx + R] - su[ly + R + 1 + k][lx + R]);
            }
            const T bsum = bxn + byn;
            T rhs = -bxn * byn * u + pc2[b][c] * ((uxx + uyy) * idx2 + (dwx + dwy) * idx1);
            if (i == P->src_i && j == P->src_j) rhs += sig;
            const T um = pum[b][c];
            T up;
            if (variant == 2) {
                // (u^{n+1} - u^n)(1 + b dt/2) = d^n (1 - b dt/2) + dt^2 rhs, with d^n = um
                const T hb = T(0.5) * bsum * dt;
                const T dn = (um * (T(1) - hb) + dt * dt * rhs) / (T(1) + hb);
                Cn[fstr + o] = dn;
                up = u + dn;
            } else {
                const T inv_dt2 = T(1) / (dt * dt), inv_2dt = T(1) / (T(2) * dt);
                up = ((T(2) * u - um) * inv_dt2 + bsum * um * inv_2dt + rhs) / (inv_dt2 + bsum * inv_2dt);
            }
            T wxp = T(0), wyp = T(0);
            if (i < nx - 1) {
                const T gx = (byn - bxh) * dux * idx1;
                wxp = variant != 1 ? ((T(1) - bxh * dt) * pwxm[b][c] + T(2) * dt * gx) / (T(1) + bxh * dt)
                                   : pwxm[b][c] + T(2) * dt * (-bxh * swx[ly][lx + R] + gx);
            }
            if (j < ny - 1) {
                const T gy = (bxn - byh) * duy * idx1;
                wyp = variant != 1 ? ((T(1) - byh * dt) * pwym[b][c] + T(2) * dt * gy) / (T(1) + byh * dt)
                                   : pwym[b][c] + T(2) * dt * (-byh * swy[ly + R][lx] + gy);
            }
            Pn[o] = up;
            Pn[2 * fstr + o] = wxp;
            Pn[3 * fstr + o] = wyp;
        }
}

// --------------------------------------------------------------------------------------
void launch_stage(int precision, int R, int nblocks, const ProblemDev* probs,
                  const int* tile_prob, const StageArgs& a, cudaStream_t s) {
    const dim3 block(TPX, TPY);
    if (nblocks <= 0) return;
    if (precision == 0) {
        if (R == 4) {
            if (a.transpose) stage_kernel<float, 4, true><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
            else stage_kernel<float, 4, false><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
        } else {
            if (a.transpose) stage_kernel<float, 2, true><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
            else stage_kernel<float, 2, false><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
        }
    } else {
        if (R == 4) {
            if (a.transpose) stage_kernel<double, 4, true><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
            else stage_kernel<double, 4, false><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
        } else {
            if (a.transpose) stage_kernel<double, 2, true><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
            else stage_kernel<double, 2, false><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
        }
    }
}

// --------------------------------------------------------------------------------------
// Pointwise parts of the discrete adjoint of the leap-frog step (averaged damping of w).
// One step maps z^n = (u^n, u^{n-1}, w^n, w^{n-1}) to z^{n+1} with
//   u^{n+1} = s (2u^n/dt^2 + (b/(2dt) - 1/dt^2) u^{n-1} + H_vu u^n + H_vw w^n + f),
//   w^{n+1} = ((1 - beta dt) w^{n-1} + 2 dt H_wu u^n) / (1 + beta dt),
// s = 1 / (1/dt^2 + b/(2dt)), b = b_x + b_y at the node, beta the w row's own damping, and
// H_vu, H_vw, H_wu blocks of H (Eq. 1).  Its transpose needs one H^T pass on
// q = (0, s lam_u, 2 dt lam_w / (1 + beta dt)):
//   lam_u'   = (H^T q)_u + (2/dt^2) s lam_u + lam_um,
//   lam_um'  = s (b/(2dt) - 1/dt^2) lam_u,
//   lam_w'   = (H^T q)_w + beta q_w + lam_wm        ((H^T q)_w holds -beta q_w),
//   lam_wm'  = (1 - beta dt) / (1 + beta dt) lam_w.
// Layout: vector 0 of a problem holds (lam_u, lam_um, lam_wx, lam_wy) (lam_um in the v field),
// a1 + shot * vec_stride holds lam_wm in its w fields.  mode 0 writes q into vector `qv`;
// mode 1 applies the update above with (H^T q) in vector `yv`.
// --------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
leapfrog_adjoint_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tile_prob,
                        int mode, int qv, int yv, void* a1_base, double dt_d) {
    const int pid = tile_prob[blockIdx.x];
    const ProblemDev* P = probs + pid;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = P->nx, ny = P->ny, pitch = P->pitch, pml = P->pml;
    const bool fs = P->fs != 0;
    const int lt = blockIdx.x - P->tile_base;
    const int x0 = (lt % P->tiles_x) * BX, y0 = (lt / P->tiles_x) * BY;
    const long long fstr = P->field_stride;
    const T beta0 = (T)P->beta0, inv_pml = (T)P->inv_pml;
    const T dt = (T)dt_d;
    T* L0 = vec_ptr<T>(P, 0);
    T* L1 = (T*)a1_base + (long long)P->shot * P->vec_stride;
#pragma unroll
    for (int b = 0; b < VY; ++b)
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int i = x0 + tx + c * TPX, j = y0 + ty + b * TPY;
            if (i >= nx || j >= ny) continue;
            const long long o = (long long)j * pitch + i;
            const T bxn = damp<T>(beta0, inv_pml, T(min(i + 1, nx - i)), pml);
            const T byn = damp<T>(beta0, inv_pml, fs ? T(ny - j) : T(min(j + 1, ny - j)), pml);
            const T bxh = damp<T>(beta0, inv_pml, min(T(i) + T(1.5), T(nx - i) - T(0.5)), pml);
            const T byh = damp<T>(beta0, inv_pml,
                                  fs ? (T(ny - j) - T(0.5)) : min(T(j) + T(1.5), T(ny - j) - T(0.5)),
                                  pml);
            const T bsum = bxn + byn;
            const T inv_dt2 = T(1) / (dt * dt), inv_2dt = T(1) / (T(2) * dt);
            const T sn = T(1) / (inv_dt2 + bsum * inv_2dt);
            const bool hx = i < nx - 1, hy = j < ny - 1;
            const T lu = L0[o], lwx = hx ? L0[2 * fstr + o] : T(0), lwy = hy ? L0[3 * fstr + o] : T(0);
            if (mode == 0) {
                T* Q = vec_ptr<T>(P, qv);
                Q[o] = T(0);
                Q[fstr + o] = sn * lu;
                Q[2 * fstr + o] = hx ? T(2) * dt * lwx / (T(1) + bxh * dt) : T(0);
                Q[3 * fstr + o] = hy ? T(2) * dt * lwy / (T(1) + byh * dt) : T(0);
            } else {
                const T* Y = vec_ptr<T>(P, yv);
                // every operand is loaded before the first store (one memory round trip)
                const T lum = L0[fstr + o], yu = Y[o];
                const T ywx = hx ? Y[2 * fstr + o] : T(0), l1x = hx ? L1[2 * fstr + o] : T(0);
                const T ywy = hy ? Y[3 * fstr + o] : T(0), l1y = hy ? L1[3 * fstr + o] : T(0);
                L0[o] = yu + T(2) * inv_dt2 * sn * lu + lum;
                L0[fstr + o] = sn * (bsum * inv_2dt - inv_dt2) * lu;
                if (hx) {
                    const T qx = T(2) * dt * lwx / (T(1) + bxh * dt);
                    L0[2 * fstr + o] = ywx + bxh * qx + l1x;
                    L1[2 * fstr + o] = (T(1) - bxh * dt) / (T(1) + bxh * dt) * lwx;
                }
                if (hy) {
                    const T qy = T(2) * dt * lwy / (T(1) + byh * dt);
                    L0[3 * fstr + o] = ywy + byh * qy + l1y;
                    L1[3 * fstr + o] = (T(1) - byh * dt) / (T(1) + byh * dt) * lwy;
                }
            }
        }
}

void launch_leapfrog_adjoint(int precision, int nblocks, const ProblemDev* probs, const int* tile_prob,
                             int mode, int qv, int yv, void* a1_base, double dt, cudaStream_t s) {
    const dim3 block(TPX, TPY);
    if (nblocks <= 0) return;
    if (precision == 0)
        leapfrog_adjoint_kernel<float><<<nblocks, block, 0, s>>>(probs, tile_prob, mode, qv, yv, a1_base, dt);
    else
        leapfrog_adjoint_kernel<double><<<nblocks, block, 0, s>>>(probs, tile_prob, mode, qv, yv, a1_base, dt);
}

void launch_leapfrog(int precision, int R, int nblocks, const ProblemDev* probs,
                     const int* tile_prob, int cur, int prev, int variant, double dt,
                     cudaStream_t s) {
    const dim3 block(TPX, TPY);
    if (nblocks <= 0) return;
    if (precision == 0) {
        if (R == 4) leapfrog_kernel<float, 4><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
        else leapfrog_kernel<float, 2><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
    } else {
        if (R == 4) leapfrog_kernel<double, 4><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
        else leapfrog_kernel<double, 2><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
    }
}

}  // namespace ewv
