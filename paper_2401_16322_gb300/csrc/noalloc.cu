// Allocation-free Faber step (ewv_faber_step_noalloc in include/ewave.h).
//
// Some callers cannot call cudaMalloc at all: code that runs inside a memory pool owned by
// someone else, embedded or certified environments that forbid run-time allocation, or a
// host process that must not grow the device heap while other work holds it.  For them
// this file provides one entry point that needs no handle and allocates nothing.  Every
// buffer the step needs beyond the caller's state and c^2 -- the two Faber work vectors,
// the problem descriptor, the tile list, the per-step source scalars, the clock and the
// coefficients -- lives in one file-scope device array, g_noalloc_scratch, of a fixed
// size.  Every GPU that loads the library holds that array until the process exits.
//
// Host code must not use the array's name as a device address: on the host it denotes a
// host-side shadow symbol.  The first call on each device (with that device current)
// obtains the real device address with cudaGetSymbolAddress and caches it; that first call
// should come before any stream capture.  All calls share the array and it keeps the last
// call's contents; everything a step reads from it is written earlier in the same call,
// so nothing is cleared.  Calls whose GPU work overlaps (two streams, or two host threads)
// race on the array.
#include <mutex>

#include "../../include/ewave.h"
#include "ewave_internal.cuh"

namespace ewv {

int ensure_tables_current_device();

namespace {

constexpr size_t kMetaBytes = 256 * 1024;                       // descriptors, scalars, tiles
constexpr size_t kVecBytes = (size_t)4 * EWV_NOALLOC_MAX_FIELD_ELEMS * sizeof(float);
constexpr size_t kScratchBytes = kMetaBytes + 2 * kVecBytes;     // 16 MB + 256 KB
constexpr int kMaxTiles = 16384;

// meta layout (bytes)
constexpr size_t OFF_DESC = 0;                                   // ProblemDev
constexpr size_t OFF_SIGMA = 1024;                               // MAX_SIGMA doubles
constexpr size_t OFF_CLK = OFF_SIGMA + MAX_SIGMA * 8;            // 4 long long
constexpr size_t OFF_TCLK = OFF_CLK + 64;                        // 2 doubles
constexpr size_t OFF_COEF = OFF_TCLK + 64;                       // MAX_DEG + 1 doubles
constexpr size_t OFF_KRY = ((OFF_COEF + (MAX_DEG + 1) * 8 + 255) / 256) * 256;
constexpr size_t OFF_TILES = ((OFF_KRY + KRY_STRIDE * 8 + 255) / 256) * 256;
static_assert(OFF_TILES + kMaxTiles * sizeof(int) <= kMetaBytes, "meta region too small");
static_assert(sizeof(ProblemDev) <= OFF_SIGMA, "descriptor slot too small");

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

}  // namespace

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void noalloc_init_kernel(ProblemDev P, ProblemDev* desc, int* tiles, int ntiles) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *desc = P;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
        tiles[t] = 0;
}

static int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EWV_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return EWV_ERR_CUDA;
        if (ensure_tables_current_device() != 0) return EWV_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return EWV_OK;
}

}  // namespace ewv

using namespace ewv;

extern "C" int ewv_faber_step_noalloc(const ewv_noalloc_faber_args* a, float* state,
                                      const float* c2, double t, double dt, int degree,
                                      int nsteps, void* stream) {
    if (!a || !state || !c2) return EWV_ERR_INVALID_ARG;
    if (a->nx < 2 || a->ny < 2 || a->pitch < a->nx || (a->pitch % 32) != 0 || !(a->dx > 0) ||
        (a->fd_order != 4 && a->fd_order != 8) || a->pml_width < 0 || a->beta0 < 0 ||
        (a->free_surface && a->fd_order != 8) || degree < 1 || degree > MAX_DEG || nsteps < 0 ||
        !(dt > 0) || !(a->gamma > 0) || a->src_taylor_p < 1 || a->src_taylor_p > MAX_P)
        return EWV_ERR_INVALID_ARG;
    if (a->has_source && (a->src_i < 0 || a->src_i >= a->nx || a->src_j < 0 || a->src_j >= a->ny))
        return EWV_ERR_INVALID_ARG;
    if ((long long)a->ny * a->pitch > EWV_NOALLOC_MAX_FIELD_ELEMS) return EWV_ERR_BAD_SIZE_OR_ALIGNMENT;
    const int tiles_x = (a->nx + BX - 1) / BX, tiles_y = (a->ny + BY - 1) / BY;
    if (tiles_x * tiles_y > kMaxTiles) return EWV_ERR_BAD_SIZE_OR_ALIGNMENT;
    if (((uintptr_t)state & 15u) || ((uintptr_t)c2 & 15u)) return EWV_ERR_BAD_SIZE_OR_ALIGNMENT;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != EWV_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* b = static_cast<unsigned char*>(base);

    ProblemDev P{};
    P.nx = a->nx;
    P.ny = a->ny;
    P.pitch = a->pitch;
    P.fs = a->free_surface ? 1 : 0;
    P.nz = 1;
    P.nfields = 4;
    P.pml = a->pml_width;
    P.has_src = a->has_source ? 1 : 0;
    P.src_i = a->has_source ? a->src_i : -1;
    P.src_j = a->has_source ? a->src_j : -1;
    P.nrec = 0;
    P.tiles_x = tiles_x;
    P.tiles_y = tiles_y;
    P.ntiles = tiles_x * tiles_y;
    P.tile_base = 0;
    P.p = a->src_taylor_p;
    P.beta0 = a->beta0;
    P.inv_dx = 1.0 / a->dx;
    P.inv_dx2 = 1.0 / (a->dx * a->dx);
    P.inv_pml = a->pml_width > 0 ? 1.0 / a->pml_width : 0.0;
    P.f_peak = a->f_peak;
    P.t0 = a->t0;
    P.amp = a->amp;
    P.field_stride = (long long)a->ny * a->pitch;
    P.vec_stride = 4 * P.field_stride;
    P.state = state;
    P.work = b + kMetaBytes;
    P.c2 = c2;
    P.sigma = reinterpret_cast<double*>(b + OFF_SIGMA);
    P.rec_off = nullptr;
    P.seismo = nullptr;
    P.kry = reinterpret_cast<double*>(b + OFF_KRY);
    P.clk = reinterpret_cast<long long*>(b + OFF_CLK);
    P.tclk = reinterpret_cast<double*>(b + OFF_TCLK);
    P.tmaps = nullptr;
    ProblemDev* d_desc = reinterpret_cast<ProblemDev*>(b + OFF_DESC);
    int* d_tiles = reinterpret_cast<int*>(b + OFF_TILES);
    double* d_coef = reinterpret_cast<double*>(b + OFF_COEF);

    noalloc_init_kernel<<<32, 256, 0, s>>>(P, d_desc, d_tiles, P.ntiles);
    // Faber coefficients of exp(dt z) on the ellipse (FP64, on the GPU), read back once.
    double coef[MAX_DEG + 1];
    launch_faber_coeffs(dt, a->gamma, a->c0, a->c1, degree, d_coef, s);
    if (cudaMemcpyAsync(coef, d_coef, sizeof(double) * (degree + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return EWV_ERR_CUDA;
    const double g = a->gamma, c0 = a->c0, c1 = a->c1;
    const int R = a->fd_order / 2;
    launch_set_clock(d_desc, 1, t, dt, s);
    for (int n = 0; n < nsteps; ++n) {
        launch_prologue(d_desc, 1, /*PRO_FABER*/ 1, degree, g, c0, c1, s);
        StageArgs st{};
        st.u = st.a = st.y_out = st.acc_out = st.d = -1;
        st.src_slot = -1;
        st.x_scale_slot = -1;
        st.cx = -c0;
        st.ch = 1.0 / g;
        st.ck = 1.0;
        // degree 1: p_1 -> work 1, a_0 x + a_1 p_1 -> work 2
        st.x = 0;
        st.y_out = 1;
        st.acc_out = 2;
        st.src_slot = 0;
        st.cay = coef[1];
        st.cax = coef[0];
        launch_stage(0, R, P.ntiles, d_desc, d_tiles, st, s);
        if (degree == 1) {
            PointArgs pa{};
            pa.mode = 3;
            pa.src = 2;
            pa.dst = 0;
            pa.fmask = 0xF;
            launch_point(0, P.ntiles, d_desc, d_tiles, pa, s);
        }
        for (int j = 2; j <= degree; ++j) {
            StageArgs sj{};
            sj.u = sj.a = sj.y_out = sj.acc_out = sj.d = -1;
            sj.x_scale_slot = -1;
            sj.cx = -c0;
            sj.ch = 1.0 / g;
            sj.ck = 1.0;
            sj.ca = 1.0;
            sj.cay = coef[j];
            sj.src_slot = j - 1;
            if (j == 2) {
                sj.x = 1; sj.u = 0; sj.a = 2; sj.y_out = 2; sj.acc_out = 0; sj.cu = -2.0 * c1;
            } else {
                const int in = (j & 1) ? 2 : 1, out = (j & 1) ? 1 : 2;
                sj.x = in; sj.u = out; sj.a = 0; sj.y_out = out; sj.acc_out = 0; sj.cu = -c1;
            }
            launch_stage(0, R, P.ntiles, d_desc, d_tiles, sj, s);
        }
        // advance the step clock (no receivers are recorded by this entry point)
        launch_record(0, d_desc, 1, 0, s);
    }
    return cudaGetLastError() == cudaSuccess ? EWV_OK : EWV_ERR_CUDA;
}
