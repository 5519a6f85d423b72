// Three-dimensional fused stencil kernels (the 400^3 workload).
//
// Operator: the three-dimensional PML form of Eq. (1) with an auxiliary field psi (psi_t = u),
// on U = (u, v, w_x, w_y, w_z, psi):
//   (HU)_u   = v
//   (HU)_v   = -(bx by + by bz + bx bz) u - (bx + by + bz) v - bx by bz psi
//              + c^2 (u_xx + u_yy + u_zz + d_x w_x + d_y w_y + d_z w_z)
//   (HU)_w_a = (sum of the other two b's - b_a) d_a u + (product of the other two b's) d_a psi
//              - b_a w_a                                            (a = x, y, z)
//   (HU)_psi = u
// With one axis undamped and a field constant along it, the u, v and remaining w rows are
// Eq. (1) on the other two axes.  The products of two b's vanish outside the edges of the
// layer, so the psi derivatives (same half-point stencils as those of u) are read from
// global memory only where their coefficient is nonzero.
// w_x lives at (i+1/2, j, k), w_y at (i, j+1/2, k), w_z at (i, j, k+1/2), psi at the nodes.  The stencils are
// Sec. 2.1's, with zero extension beyond the grid.  z is the vertical axis, k = 0 the top.
// With a free surface, z plays the part of the 2D y axis:
//   - it points upward: d_z u at k+1/2 = sum_q s_q (u_{k-q} - u_{k+1+q}) / dx;
//   - Appendix A's rows replace u_zz at k = 0..3 and d_z u at k+1/2, k = 0..2;
//   - the Fornberg rows replace d_z w_z at k = 0..3;
//   - there is no z damping at the top.
// beta = beta0 (1 - d/delta)^2 (Sec. 2) is evaluated in registers.
//
// Layout: fields [nz][ny][pitch], field-major, as in 2D.  Decomposition:
//   - a block owns a BX x BY column tile in (x, y) and marches down KC3 planes of z;
//   - each thread keeps, for each of its VX x VY columns, a register queue of u over
//     k-R .. k+R and of w_z over k-R .. k+R-1, which supplies every z-stencil tap;
//   - the current plane of u (2D halo), w_x (x halo) and w_y (y halo) is staged in shared
//     memory for the x and y taps;
//   - pointwise operands (v, c^2 and the integrator's vectors) are read straight from global
//     memory, coalesced along x.
//
// The epilogue per field f is that of the 2D pass (kernels_stencil.cu):
//   K = cx xs X + ch xs (H X + sigma e_src),  Y = cu U + ck K,
//   ACC = ca A + cau U + cak K + cay Y + cax xs X,
// with an optional partial dot product <Y, D> finalised by the problem's last block.
#include <type_traits>

#include "ewave_internal.cuh"
#include "krylov_finalize.cuh"

namespace ewv {

namespace {

__constant__ double g3_fs_d[4 * 9 + 3 * 8 + 4 * 8];
__constant__ float g3_fs_f[4 * 9 + 3 * 8 + 4 * 8];
constexpr int FS3_UZZ = 0, FS3_UZ = 36, FS3_DWZ = 60;

template <typename T>
__device__ __forceinline__ T fs3(int off) {
    if constexpr (std::is_same<T, float>::value) return g3_fs_f[off];
    else return g3_fs_d[off];
}

template <typename T, int R>
__device__ __forceinline__ T S3(int k) {   // staggered first derivative (Eq. spatial_8th_1)
    if constexpr (R == 4) {
        return k == 0 ? T(1225.0 / 1024.0) : k == 1 ? T(-245.0 / 3072.0)
             : k == 2 ? T(49.0 / 5120.0) : T(-5.0 / 7168.0);
    } else {
        return k == 0 ? T(9.0 / 8.0) : T(-1.0 / 24.0);
    }
}
template <typename T, int R>
__device__ __forceinline__ T C3(int k) {   // centred second derivative (Eq. spatial_8th_2)
    if constexpr (R == 4) {
        return k == 0 ? T(-205.0 / 72.0) : k == 1 ? T(8.0 / 5.0) : k == 2 ? T(-1.0 / 5.0)
             : k == 3 ? T(8.0 / 315.0) : T(-1.0 / 560.0);
    } else {
        return k == 0 ? T(-5.0 / 2.0) : k == 1 ? T(4.0 / 3.0) : T(-1.0 / 12.0);
    }
}

template <typename T>
__device__ __forceinline__ T damp3(T beta0, T inv_pml, T d, int pml) {
    if (pml <= 0) return T(0);
    const T r = T(1) - d * inv_pml;
    return (d <= T(pml)) ? beta0 * r * r : T(0);
}

template <typename T>
__device__ __forceinline__ T* vec3(const ProblemDev* P, int k) {
    return k == 0 ? (T*)P->state : (T*)P->work + (long long)(k - 1) * P->vec_stride;
}

// Shared per-tile geometry.
struct Tile3 {
    int x0, y0, k0, k1;
};

__device__ __forceinline__ Tile3 tile3_of(const ProblemDev* P, int lt) {
    Tile3 t;
    const int txi = lt % P->tiles_x;
    const int r = lt / P->tiles_x;
    const int tyi = r % P->tiles_y;
    const int tzi = r / P->tiles_y;
    t.x0 = txi * BX;
    t.y0 = tyi * BY;
    t.k0 = tzi * KC3;
    t.k1 = min(t.k0 + KC3, P->nz);
    return t;
}

// The derivative terms of one output point: Laplacian, divergence of w and the three
// half-point derivatives of u (all still to be scaled by 1/dx^2 or 1/dx).
template <typename T>
struct Deriv3 {
    T lap, div, dux, duy, duz;
};

// u column value at level q (0 <= q < nz) for the free-surface rows, from global memory.
template <typename T>
__device__ __forceinline__ T colv(const T* base, long long ps, int q, int nmax) {
    return q < nmax ? base[(long long)q * ps] : T(0);
}

// Half-point first derivative of psi along one axis (not yet scaled by 1/dx), read from
// global memory: p points at psi of the output's own node, `stride` is the axis stride, idx
// the node index along the axis and n its extent (zero extension).  up = true: the vertical
// axis, whose derivative at k+1/2 is sum_q s_q (psi_{k-q} - psi_{k+1+q}).
template <typename T, int R>
__device__ __forceinline__ T dpsi_half(const T* p, long long stride, int idx, int n, bool up) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const T fwd = (idx + 1 + q < n) ? p[(long long)(1 + q) * stride] : T(0);
        const T bwd = (idx - q >= 0) ? p[-(long long)q * stride] : T(0);
        s += S3<T, R>(q) * (up ? bwd - fwd : fwd - bwd);
    }
    return s;
}
// d_z psi at half level k+1/2 near a free surface (k < 3): the Appendix A rows.
template <typename T>
__device__ __forceinline__ T dpsi_fs(const T* col, long long ps, int k, int nz) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) s += fs3<T>(FS3_UZ + k * 8 + q) * colv(col, ps, q, nz);
    return s;
}

// The psi terms of one output point: the products of two damping coefficients times the
// psi derivatives (scaled by 1/dx), zero where the product vanishes.
template <typename T, int R>
__device__ __forceinline__ void psi_terms(const T* psi_c, long long pitch, long long ps, int i,
                                          int j, int k, int nx, int ny, int nz, bool fs,
                                          T pyz, T pxz, T pxy, T idx1, T& gx, T& gy, T& gz) {
    gx = (pyz != T(0) && i < nx - 1) ? pyz * dpsi_half<T, R>(psi_c, 1, i, nx, false) * idx1 : T(0);
    gy = (pxz != T(0) && j < ny - 1) ? pxz * dpsi_half<T, R>(psi_c, pitch, j, ny, false) * idx1 : T(0);
    gz = T(0);
    if (pxy != T(0) && k < nz - 1) {
        const T d = (fs && k < 3) ? dpsi_fs<T>(psi_c - (long long)k * ps, ps, k, nz)
                                  : dpsi_half<T, R>(psi_c, ps, k, nz, true);
        gz = pxy * d * idx1;
    }
}

template <typename T, int R>
__device__ __forceinline__ Deriv3<T> derivs3(const T (&su)[BY + 2 * R][BX + 2 * R],
                                             const T (&swx)[BY][BX + 2 * R],
                                             const T (&swy)[BY + 2 * R][BX], const T* uq,
                                             const T* wzq, int lx, int ly, int k, bool fs_top,
                                             const T* ucol, const T* wzcol, long long ps, int nz) {
    Deriv3<T> d;
    const T u = uq[R];
    T uxx = C3<T, R>(0) * u, uyy = C3<T, R>(0) * u;
#pragma unroll
    for (int q = 1; q <= R; ++q) {
        uxx += C3<T, R>(q) * (su[ly + R][lx + R + q] + su[ly + R][lx + R - q]);
        uyy += C3<T, R>(q) * (su[ly + R + q][lx + R] + su[ly + R - q][lx + R]);
    }
    T uzz, dwz, duz;
    if (fs_top && k < 4) {
        uzz = T(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) uzz += fs3<T>(FS3_UZZ + k * 9 + q) * colv(ucol, ps, q, nz);
        dwz = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) dwz += fs3<T>(FS3_DWZ + k * 8 + q) * colv(wzcol, ps, q, nz - 1);
    } else {
        uzz = C3<T, R>(0) * u;
#pragma unroll
        for (int q = 1; q <= R; ++q) uzz += C3<T, R>(q) * (uq[R + q] + uq[R - q]);
        dwz = T(0);
#pragma unroll
        for (int q = 0; q < R; ++q) dwz += S3<T, R>(q) * (wzq[R - 1 - q] - wzq[R + q]);
    }
    if (fs_top && k < 3) {
        duz = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) duz += fs3<T>(FS3_UZ + k * 8 + q) * colv(ucol, ps, q, nz);
    } else {
        duz = T(0);
#pragma unroll
        for (int q = 0; q < R; ++q) duz += S3<T, R>(q) * (uq[R - q] - uq[R + 1 + q]);
    }
    T dwx = T(0), dwy = T(0), dux = T(0), duy = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        dwx += S3<T, R>(q) * (swx[ly][lx + R + q] - swx[ly][lx + R - 1 - q]);
        dwy += S3<T, R>(q) * (swy[ly + R + q][lx] - swy[ly + R - 1 - q][lx]);
        dux += S3<T, R>(q) * (su[ly + R][lx + R + 1 + q] - su[ly + R][lx + R - q]);
        duy += S3<T, R>(q) * (su[ly + R + 1 + q][lx + R] - su[ly + R - q][lx + R]);
    }
    d.lap = uxx + uyy + uzz;
    d.div = dwx + dwy + dwz;
    d.dux = dux;
    d.duy = duy;
    d.duz = duz;
    return d;
}

// Stage the current plane k of u (2D halo, interior from the register queues), w_x (x halo)
// and w_y (y halo) into shared memory.  Zero outside the grid (zero extension).
template <typename T, int R>
__device__ __forceinline__ void stage_plane3(T (&su)[BY + 2 * R][BX + 2 * R],
                                             T (&swx)[BY][BX + 2 * R], T (&swy)[BY + 2 * R][BX],
                                             const T* Xu, const T* Xwx, const T* Xwy,
                                             const T (&center)[VY][VX], int x0, int y0, int nx,
                                             int ny, int pitch, int tid) {
    constexpr int SW = BX + 2 * R, SH = BY + 2 * R;
    for (int idx = tid; idx < SH * SW; idx += NTHREADS) {
        const int r = idx / SW, c = idx - r * SW;
        if (r >= R && r < BY + R && c >= R && c < BX + R) continue;   // interior: from queue
        const int gx = x0 - R + c, gy = y0 - R + r;
        su[r][c] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? Xu[(long long)gy * pitch + gx] : T(0);
    }
    const int tx = tid % TPX, ty = tid / TPX;
#pragma unroll
    for (int b = 0; b < VY; ++b)
#pragma unroll
        for (int c = 0; c < VX; ++c) su[ty + b * TPY + R][tx + c * TPX + R] = center[b][c];
    for (int idx = tid; idx < BY * SW; idx += NTHREADS) {
        const int r = idx / SW, c = idx - r * SW;
        const int gx = x0 - R + c, gy = y0 + r;
        swx[r][c] = (gx >= 0 && gx < nx - 1 && gy < ny) ? Xwx[(long long)gy * pitch + gx] : T(0);
    }
    for (int idx = tid; idx < SH * BX; idx += NTHREADS) {
        const int r = idx / BX, c = idx - r * BX;
        const int gx = x0 + c, gy = y0 - R + r;
        swy[r][c] = (gx < nx && gy >= 0 && gy < ny - 1) ? Xwy[(long long)gy * pitch + gx] : T(0);
    }
}

// --------------------------------------------------------------------------------------
// Stage kernel: one fused pass of an integrator (forward operator only).
// --------------------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(NTHREADS)
stage3d_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tile_prob,
               StageArgs a) {
    __shared__ T su[BY + 2 * R][BX + 2 * R];
    __shared__ T swx[BY][BX + 2 * R];
    __shared__ T swy[BY + 2 * R][BX];
    __shared__ double red[NTHREADS / 32];
    __shared__ int s_last;

    const int pid = tile_prob[blockIdx.x];
    const ProblemDev* P = probs + pid;
    if (a.fin_mode != FIN_NONE && P->kry[KRY_ACTIVE] == 0.0) return;   // Arnoldi stopped

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TPX + tx;
    const int nx = P->nx, ny = P->ny, nz = P->nz, pitch = P->pitch, pml = P->pml;
    const bool fs = P->fs != 0;
    const Tile3 tl = tile3_of(P, blockIdx.x - P->tile_base);
    const long long fstr = P->field_stride;
    const long long ps = (long long)ny * pitch;
    const T beta0 = (T)P->beta0, inv_pml = (T)P->inv_pml;
    const T idx1 = (T)P->inv_dx, idx2 = (T)P->inv_dx2;

    const T* X = vec3<T>(P, a.x);
    const T* C2 = (const T*)P->c2;
    const T* U = a.u >= 0 ? vec3<T>(P, a.u) : nullptr;
    const T* A = a.a >= 0 ? vec3<T>(P, a.a) : nullptr;
    T* Y = a.y_out >= 0 ? vec3<T>(P, a.y_out) : nullptr;
    T* ACC = a.acc_out >= 0 ? vec3<T>(P, a.acc_out) : nullptr;
    const T* D = a.d >= 0 ? vec3<T>(P, a.d) : nullptr;
    const T cx = (T)a.cx, ch = (T)a.ch, cu = (T)a.cu, ck = (T)a.ck, ca = (T)a.ca;
    const T cau = (T)a.cau, cak = (T)a.cak, cay = (T)a.cay, cax = (T)a.cax;
    const T xs = a.x_scale_slot >= 0 ? (T)P->kry[a.x_scale_slot] : T(1);
    const T sig = (a.src_slot >= 0 && P->has_src) ? (T)P->sigma[a.src_slot] : T(0);

    // register queues: uq[..][0..2R] = u(k-R .. k+R), wq[..][0..2R-1] = w_z(k-R .. k+R-1)
    T uq[VY][VX][2 * R + 1];
    T wq[VY][VX][2 * R];
#pragma unroll
    for (int b = 0; b < VY; ++b)
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int i = tl.x0 + tx + c * TPX, j = tl.y0 + ty + b * TPY;
            const bool in = i < nx && j < ny;
            const long long o = (long long)j * pitch + i;
#pragma unroll
            for (int q = 0; q < 2 * R; ++q) {
                const int ku = tl.k0 - R + q;
                uq[b][c][q + 1] = (in && ku >= 0 && ku < nz) ? X[ku * ps + o] : T(0);
            }
#pragma unroll
            for (int q = 0; q < 2 * R - 1; ++q) {
                const int kw = tl.k0 - R + q;
                wq[b][c][q + 1] = (in && kw >= 0 && kw < nz - 1) ? X[4 * fstr + kw * ps + o] : T(0);
            }
        }

    float dotf = 0.f;
    double dotd = 0.0;
    for (int k = tl.k0; k < tl.k1; ++k) {
        T center[VY][VX];
#pragma unroll
        for (int b = 0; b < VY; ++b)
#pragma unroll
            for (int c = 0; c < VX; ++c) {
                const int i = tl.x0 + tx + c * TPX, j = tl.y0 + ty + b * TPY;
                const bool in = i < nx && j < ny;
                const long long o = (long long)j * pitch + i;
#pragma unroll
                for (int q = 0; q < 2 * R; ++q) uq[b][c][q] = uq[b][c][q + 1];
#pragma unroll
                for (int q = 0; q < 2 * R - 1; ++q) wq[b][c][q] = wq[b][c][q + 1];
                const int ku = k + R, kw = k + R - 1;
                uq[b][c][2 * R] = (in && ku < nz) ? X[ku * ps + o] : T(0);
                wq[b][c][2 * R - 1] = (in && kw < nz - 1) ? X[4 * fstr + kw * ps + o] : T(0);
                center[b][c] = uq[b][c][R];
            }
        __syncthreads();   // previous plane's shared reads are done
        stage_plane3<T, R>(su, swx, swy, X + k * ps, X + 2 * fstr + k * ps, X + 3 * fstr + k * ps,
                           center, tl.x0, tl.y0, nx, ny, pitch, tid);
        __syncthreads();
        const bool fs_top = fs && k < 4;
        const T bzn = damp3<T>(beta0, inv_pml, fs ? T(nz - k) : T(min(k + 1, nz - k)), pml);
        const T bzh = damp3<T>(beta0, inv_pml,
                               fs ? (T(nz - k) - T(0.5)) : min(T(k) + T(1.5), T(nz - k) - T(0.5)), pml);
#pragma unroll
        for (int b = 0; b < VY; ++b)
#pragma unroll
            for (int c = 0; c < VX; ++c) {
                const int lx = tx + c * TPX, ly = ty + b * TPY;
                const int i = tl.x0 + lx, j = tl.y0 + ly;
                if (i >= nx || j >= ny) continue;
                const long long o = (long long)k * ps + (long long)j * pitch + i;
                const long long oc = (long long)j * pitch + i;
                const Deriv3<T> dv = derivs3<T, R>(su, swx, swy, uq[b][c], wq[b][c], lx, ly, k,
                                                   fs_top, X + oc, X + 4 * fstr + oc, ps, nz);
                const T bxn = damp3<T>(beta0, inv_pml, T(min(i + 1, nx - i)), pml);
                const T byn = damp3<T>(beta0, inv_pml, T(min(j + 1, ny - j)), pml);
                const T bxh = damp3<T>(beta0, inv_pml, min(T(i) + T(1.5), T(nx - i) - T(0.5)), pml);
                const T byh = damp3<T>(beta0, inv_pml, min(T(j) + T(1.5), T(ny - j) - T(0.5)), pml);
                const T c2 = C2[o];
                const T xu = uq[b][c][R];
                const T xv = X[fstr + o];
                const T xwx = swx[ly][lx + R];
                const T xwy = swy[ly + R][lx];
                const T xwz = wq[b][c][R];
                const T xpsi = X[5 * fstr + o];
                T gpx, gpy, gpz;
                psi_terms<T, R>(X + 5 * fstr + o, pitch, ps, i, j, k, nx, ny, nz, fs, byn * bzn,
                                bxn * bzn, bxn * byn, idx1, gpx, gpy, gpz);
                T hv = -(bxn * byn + byn * bzn + bxn * bzn) * xu - (bxn + byn + bzn) * xv
                       - bxn * byn * bzn * xpsi + c2 * (dv.lap * idx2 + dv.div * idx1);
                if (i == P->src_i && j == P->src_j && k == P->src_k) hv += sig;
                const T hwx = (i < nx - 1) ? (byn + bzn - bxh) * dv.dux * idx1 + gpx - bxh * xwx : T(0);
                const T hwy = (j < ny - 1) ? (bxn + bzn - byh) * dv.duy * idx1 + gpy - byh * xwy : T(0);
                const T hwz = (k < nz - 1) ? (bxn + byn - bzh) * dv.duz * idx1 + gpz - bzh * xwz : T(0);
                const T xf[6] = {xu, xv, xwx, xwy, xwz, xpsi};
                const T hf[6] = {xv, hv, hwx, hwy, hwz, xu};
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    const bool pad = (f == 2 && i >= nx - 1) || (f == 3 && j >= ny - 1) ||
                                     (f == 4 && k >= nz - 1);
                    const long long of = f * fstr + o;
                    // operands first: Y may alias U or A, and ACC may alias A or U
                    const T uf = U ? U[of] : T(0);
                    const T ain = A ? A[of] : T(0);
                    const T kf = cx * xs * xf[f] + ch * xs * hf[f];
                    const T yf = pad ? T(0) : (cu * uf + ck * kf);
                    const T af = ca * ain + cau * uf + cak * kf + cay * yf + cax * xs * xf[f];
                    if (Y) Y[of] = yf;
                    if (ACC) ACC[of] = pad ? T(0) : af;
                    if (D && !pad) {
                        const T dd = D[of];
                        if constexpr (std::is_same<T, float>::value) dotf = fmaf(yf, dd, dotf);
                        else dotd = fma(yf, dd, dotd);
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
// Leap-frog kernel (Sec. 3.1's scheme on the 3D system).  Vectors `cur` (level n) and
// `prev` (level n-1) use fields 0 (u), 2, 3, 4 (w_x, w_y, w_z) and 5 (psi); level n+1
// overwrites prev.  Damping of u_t centred; damping of w time-averaged (variant 0) or
// explicit (variant 1); psi^{n+1} = psi^n + dt (u^n + u^{n+1}) / 2 (psi^{n-1} is not used).
// --------------------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(NTHREADS)
leapfrog3d_kernel(const ProblemDev* __restrict__ probs, const int* __restrict__ tile_prob,
                  int cur, int prev, int variant, double dt_d) {
    __shared__ T su[BY + 2 * R][BX + 2 * R];
    __shared__ T swx[BY][BX + 2 * R];
    __shared__ T swy[BY + 2 * R][BX];
    const int pid = tile_prob[blockIdx.x];
    const ProblemDev* P = probs + pid;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TPX + tx;
    const int nx = P->nx, ny = P->ny, nz = P->nz, pitch = P->pitch, pml = P->pml;
    const bool fs = P->fs != 0;
    const Tile3 tl = tile3_of(P, blockIdx.x - P->tile_base);
    const long long fstr = P->field_stride;
    const long long ps = (long long)ny * pitch;
    const T beta0 = (T)P->beta0, inv_pml = (T)P->inv_pml;
    const T idx1 = (T)P->inv_dx, idx2 = (T)P->inv_dx2;
    const T dt = (T)dt_d;
    const T* Cn = vec3<T>(P, cur);
    T* Pn = vec3<T>(P, prev);
    const T* C2 = (const T*)P->c2;
    const T sig = P->has_src ? (T)P->sigma[0] : T(0);

    T uq[VY][VX][2 * R + 1];
    T wq[VY][VX][2 * R];
#pragma unroll
    for (int b = 0; b < VY; ++b)
#pragma unroll
        for (int c = 0; c < VX; ++c) {
            const int i = tl.x0 + tx + c * TPX, j = tl.y0 + ty + b * TPY;
            const bool in = i < nx && j < ny;
            const long long o = (long long)j * pitch + i;
#pragma unroll
            for (int q = 0; q < 2 * R; ++q) {
                const int ku = tl.k0 - R + q;
                uq[b][c][q + 1] = (in && ku >= 0 && ku < nz) ? Cn[ku * ps + o] : T(0);
            }
#pragma unroll
            for (int q = 0; q < 2 * R - 1; ++q) {
                const int kw = tl.k0 - R + q;
                wq[b][c][q + 1] = (in && kw >= 0 && kw < nz - 1) ? Cn[4 * fstr + kw * ps + o] : T(0);
            }
        }
    for (int k = tl.k0; k < tl.k1; ++k) {
        T center[VY][VX];
#pragma unroll
        for (int b = 0; b < VY; ++b)
#pragma unroll
            for (int c = 0; c < VX; ++c) {
                const int i = tl.x0 + tx + c * TPX, j = tl.y0 + ty + b * TPY;
                const bool in = i < nx && j < ny;
                const long long o = (long long)j * pitch + i;
#pragma unroll
                for (int q = 0; q < 2 * R; ++q) uq[b][c][q] = uq[b][c][q + 1];
#pragma unroll
                for (int q = 0; q < 2 * R - 1; ++q) wq[b][c][q] = wq[b][c][q + 1];
                const int ku = k + R, kw = k + R - 1;
                uq[b][c][2 * R] = (in && ku < nz) ? Cn[ku * ps + o] : T(0);
                wq[b][c][2 * R - 1] = (in && kw < nz - 1) ? Cn[4 * fstr + kw * ps + o] : T(0);
                center[b][c] = uq[b][c][R];
            }
        __syncthreads();
        stage_plane3<T, R>(su, swx, swy, Cn + k * ps, Cn + 2 * fstr + k * ps, Cn + 3 * fstr + k * ps,
                           center, tl.x0, tl.y0, nx, ny, pitch, tid);
        __syncthreads();
        const bool fs_top = fs && k < 4;
        const T bzn = damp3<T>(beta0, inv_pml, fs ? T(nz - k) : T(min(k + 1, nz - k)), pml);
        const T bzh = damp3<T>(beta0, inv_pml,
                               fs ? (T(nz - k) - T(0.5)) : min(T(k) + T(1.5), T(nz - k) - T(0.5)), pml);
        const T inv_dt2 = T(1) / (dt * dt), inv_2dt = T(1) / (T(2) * dt);
#pragma unroll
        for (int b = 0; b < VY; ++b)
#pragma unroll
            for (int c = 0; c < VX; ++c) {
                const int lx = tx + c * TPX, ly = ty + b * TPY;
                const int i = tl.x0 + lx, j = tl.y0 + ly;
                if (i >= nx || j >= ny) continue;
                const long long o = (long long)k * ps + (long long)j * pitch + i;
                const long long oc = (long long)j * pitch + i;
                const Deriv3<T> dv = derivs3<T, R>(su, swx, swy, uq[b][c], wq[b][c], lx, ly, k,
                                                   fs_top, Cn + oc, Cn + 4 * fstr + oc, ps, nz);
                const T bxn = damp3<T>(beta0, inv_pml, T(min(i + 1, nx - i)), pml);
                const T byn = damp3<T>(beta0, inv_pml, T(min(j + 1, ny - j)), pml);
                const T bxh = damp3<T>(beta0, inv_pml, min(T(i) + T(1.5), T(nx - i) - T(0.5)), pml);
                const T byh = damp3<T>(beta0, inv_pml, min(T(j) + T(1.5), T(ny - j) - T(0.5)), pml);
                const T u = uq[b][c][R];
                const T bsum = bxn + byn + bzn;
                const T psi = Cn[5 * fstr + o];
                T gp[3];
                psi_terms<T, R>(Cn + 5 * fstr + o, pitch, ps, i, j, k, nx, ny, nz, fs, byn * bzn,
                                bxn * bzn, bxn * byn, idx1, gp[0], gp[1], gp[2]);
                T rhs = -(bxn * byn + byn * bzn + bxn * bzn) * u - bxn * byn * bzn * psi
                        + C2[o] * (dv.lap * idx2 + dv.div * idx1);
                if (i == P->src_i && j == P->src_j && k == P->src_k) rhs += sig;
                const T um = Pn[o];
                const T up = ((T(2) * u - um) * inv_dt2 + bsum * um * inv_2dt + rhs)
                             / (inv_dt2 + bsum * inv_2dt);
                T wn[3] = {T(0), T(0), T(0)};
                const bool has[3] = {i < nx - 1, j < ny - 1, k < nz - 1};
                const T bh[3] = {bxh, byh, bzh};
                const T gcoef[3] = {byn + bzn - bxh, bxn + bzn - byh, bxn + byn - bzh};
                const T du[3] = {dv.dux, dv.duy, dv.duz};
                const T wcur[3] = {swx[ly][lx + R], swy[ly + R][lx], wq[b][c][R]};
#pragma unroll
                for (int a3 = 0; a3 < 3; ++a3) {
                    if (!has[a3]) continue;
                    const T wm = Pn[(2 + a3) * fstr + o];
                    const T g = gcoef[a3] * du[a3] * idx1 + gp[a3];
                    wn[a3] = variant == 0 ? ((T(1) - bh[a3] * dt) * wm + T(2) * dt * g) / (T(1) + bh[a3] * dt)
                                          : wm + T(2) * dt * (-bh[a3] * wcur[a3] + g);
                }
                Pn[o] = up;
                Pn[2 * fstr + o] = wn[0];
                Pn[3 * fstr + o] = wn[1];
                Pn[4 * fstr + o] = wn[2];
                Pn[5 * fstr + o] = psi + T(0.5) * dt * (u + up);   // trapezoid rule for psi_t = u
            }
    }
}

}  // namespace

int upload_stencil_tables_3d(const double* fs_uzz, const double* fs_uz, const double* fs_dwz) {
    double d[92];
    float f[92];
    for (int i = 0; i < 36; ++i) d[FS3_UZZ + i] = fs_uzz[i];
    for (int i = 0; i < 24; ++i) d[FS3_UZ + i] = fs_uz[i];
    for (int i = 0; i < 32; ++i) d[FS3_DWZ + i] = fs_dwz[i];
    for (int i = 0; i < 92; ++i) f[i] = (float)d[i];
    if (cudaMemcpyToSymbol(g3_fs_d, d, sizeof(d)) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(g3_fs_f, f, sizeof(f)) != cudaSuccess) return -1;
    return 0;
}

void launch_stage3d(int precision, int R, int nblocks, const ProblemDev* probs,
                    const int* tile_prob, const StageArgs& a, cudaStream_t s) {
    const dim3 block(TPX, TPY);
    if (nblocks <= 0) return;
    if (precision == 0) {
        if (R == 4) stage3d_kernel<float, 4><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
        else stage3d_kernel<float, 2><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
    } else {
        if (R == 4) stage3d_kernel<double, 4><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
        else stage3d_kernel<double, 2><<<nblocks, block, 0, s>>>(probs, tile_prob, a);
    }
}

void launch_leapfrog3d(int precision, int R, int nblocks, const ProblemDev* probs,
                       const int* tile_prob, int cur, int prev, int variant, double dt,
                       cudaStream_t s) {
    const dim3 block(TPX, TPY);
    if (nblocks <= 0) return;
    if (precision == 0) {
        if (R == 4) leapfrog3d_kernel<float, 4><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
        else leapfrog3d_kernel<float, 2><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
    } else {
        if (R == 4) leapfrog3d_kernel<double, 4><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
        else leapfrog3d_kernel<double, 2><<<nblocks, block, 0, s>>>(probs, tile_prob, cur, prev, variant, dt);
    }
}

}  // namespace ewv
