// Host implementation of the C ABI declared in include/ewave.h.
//
// Each model owns small device metadata (per-shot source scalars, Krylov scalar blocks,
// step clocks, receiver offsets); the caller owns the grid-sized buffers.  Stepping goes
// through an Engine: the list of problems (model, shot) of one model or of a batch, the
// tile work list across all of their grids, and the per-method launch plan.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ewave.h"
#include "ewave_internal.cuh"


using namespace ewv;

namespace {
int ensure_tables();
}

namespace ewv {
int ensure_tables_current_device() { return ensure_tables(); }
}  // namespace ewv

namespace {

const char* kVersion = "ewave-gb300 0.1 (sm_103a)";

// Field mask of whole state vectors for the copy pass (bit f = field f; 2D uses bits 0..3).
constexpr int ALL_FIELDS = 0x3F;   // every field of a 2D (4) or 3D (6) vector

enum { PRO_FABER = 1, PRO_KRYLOV = 2, PRO_HORK = 3, PRO_RK32 = 4, PRO_RK44 = 5, PRO_LEAPFROG = 6,
       PRO_HORK_HORNER = 7 };
enum { FIN_NONE = 0, FIN_NORM0 = 1, FIN_MATVEC = 2, FIN_MGS = 3 };

// ---------------------------------------------------------------- stencil tables
// Appendix A free-surface rows (physical y, u_i = u(x, -i dx)), the library's own copy.
const double kFsUyy[4][9] = {
    {-3144919.0 / 352800.0, 16.0, -14.0, 112.0 / 9.0, -35.0 / 4.0, 112.0 / 25.0, -14.0 / 9.0,
     16.0 / 49.0, -1.0 / 32.0},
    {271343.0 / 156800.0, -1991.0 / 630.0, 57.0 / 40.0, 13.0 / 60.0, -109.0 / 288.0, 6.0 / 25.0,
     -11.0 / 120.0, 179.0 / 8820.0, -9.0 / 4480.0},
    {-18519.0 / 78400.0, 58.0 / 35.0, -251.0 / 90.0, 22.0 / 15.0, -1.0 / 16.0, -14.0 / 225.0,
     1.0 / 30.0, -2.0 / 245.0, 17.0 / 20160.0},
    {74801.0 / 1411200.0, -37.0 / 140.0, 67.0 / 40.0, -263.0 / 90.0, 53.0 / 32.0, -23.0 / 100.0,
     13.0 / 360.0, -1.0 / 245.0, 1.0 / 4480.0}};
const double kFsUy[3][8] = {
    {5034629.0 / 3763200.0, -23533.0 / 15360.0, 4259.0 / 15360.0, -1103.0 / 9216.0,
     151.0 / 3072.0, -1171.0 / 76800.0, 139.0 / 46080.0, -211.0 / 752640.0},
    {-363509.0 / 3763200.0, 6297.0 / 5120.0, -6147.0 / 5120.0, 211.0 / 3072.0, 3.0 / 1024.0,
     -153.0 / 25600.0, 29.0 / 15360.0, -57.0 / 250880.0},
    {4631.0 / 250880.0, -305.0 / 3072.0, 1245.0 / 1024.0, -3725.0 / 3072.0, 275.0 / 3072.0,
     -69.0 / 5120.0, 5.0 / 3072.0, -5.0 / 50176.0}};

// Finite-difference weights of the first derivative at z from values at points xs
// (Fornberg 1988: weights grow one point at a time; double precision).
void fd_weights_first(double z, const double* xs, int n, double* w_out) {
    // c[k][j]: weight of point j for derivative k (k = 0, 1)
    std::vector<double> c0(n, 0.0), c1(n, 0.0);
    double cprod = 1.0;
    double dprev = xs[0] - z;
    c0[0] = 1.0;
    for (int i = 1; i < n; ++i) {
        double prod = 1.0;
        const double dcur = xs[i] - z;
        for (int j = 0; j < i; ++j) {
            const double diff = xs[i] - xs[j];
            prod *= diff;
            if (j == i - 1) {
                c1[i] = cprod * (c0[i - 1] - dprev * c1[i - 1]) / prod;
                c0[i] = -cprod * dprev * c0[i - 1] / prod;
            }
            c1[j] = (dcur * c1[j] - c0[j]) / diff;
            c0[j] = dcur * c0[j] / diff;
        }
        cprod = prod;
        dprev = dcur;
    }
    for (int j = 0; j < n; ++j) w_out[j] = c1[j];
}

// d(w_y)/dy rows at y = -j (j = 0..3) from w_y(0) = 0 and w_y at y = -(q + 1/2), q = 0..7.
void fs_dwy_table(double out[4][8]) {
    double xs[9];
    xs[0] = 0.0;
    for (int q = 0; q < 8; ++q) xs[q + 1] = -(q + 0.5);
    for (int j = 0; j < 4; ++j) {
        double w[9];
        fd_weights_first(-(double)j, xs, 9, w);
        for (int q = 0; q < 8; ++q) out[j][q] = w[q + 1];
    }
}

int g_tables_device = -1;

int ensure_tables() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (g_tables_device == dev) return 0;
    double dwy[4][8];
    fs_dwy_table(dwy);
    if (upload_stencil_tables(8, &kFsUyy[0][0], &kFsUy[0][0], &dwy[0][0]) != 0) return -1;
    if (upload_tma_tables(&kFsUyy[0][0], &kFsUy[0][0], &dwy[0][0]) != 0) return -1;
    if (upload_stencil_tables_3d(&kFsUyy[0][0], &kFsUy[0][0], &dwy[0][0]) != 0) return -1;
    if (upload_tma3d_tables(&kFsUyy[0][0], &kFsUy[0][0], &dwy[0][0]) != 0) return -1;
    g_tables_device = dev;
    return 0;
}

// Minimum over theta of the centred second-derivative symbol.
double symbol_min(int order) {
    const double c8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
    const double c4[3] = {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0};
    const double* c = order == 8 ? c8 : c4;
    const int R = order / 2;
    double best = 1e300;
    for (int s = 0; s <= 20000; ++s) {
        const double th = M_PI * s / 20000.0;
        double v = c[0];
        for (int k = 1; k <= R; ++k) v += 2.0 * c[k] * std::cos(k * th);
        best = std::min(best, v);
    }
    return best;
}

struct Shot {
    bool has_src = false;
    int si = 0, sj = 0, sk = 0;
    double f_peak = 10.0, t0 = 0.27, amp = 1.0;
    std::vector<int> rec_off;
};

}  // namespace

struct ewv_model {
    ewv_model_desc d{};
    int R = 4, pitch = 0, elem = 4;
    int nz = 1, nfields = 4;    // 3D: nz planes and six fields (w_z and psi added)
    size_t field_elems = 0, vec_elems = 0;
    cudaStream_t stream = nullptr;
    void* state = nullptr;
    size_t state_bytes = 0;
    void* params = nullptr;
    size_t params_bytes = 0;
    void* work = nullptr;
    size_t work_bytes = 0;
    void* seismo = nullptr;
    size_t seismo_bytes = 0;
    int capacity = 0;
    double c_max = 0.0;
    bool velocity_set = false;
    std::vector<Shot> shots;
    bool ellipse_override = false;
    double eg = 0, ec0 = 0, ec1 = 0;
    int lf_variant = EWV_LEAPFROG_AVERAGED;
    int store_bf16 = 0;         // storage-precision experiment (ewv_set_storage_rounding)
    int kry_window = 0;         // Krylov orthogonalisation window (0 = full Gram-Schmidt)
    int hork_form = EWV_HORK_LOW_STORAGE;   // evaluation order of the HORK polynomial
    int kry_adjoint = EWV_KRYLOV_ADJOINT_EXACT;   // which Krylov adjoint ewv_adjoint_step runs
    bool lf_history_valid = false;
    // device metadata
    int* d_rec = nullptr;
    int* d_nrec = nullptr;      // receivers per shot
    double* d_sigma = nullptr;
    float* d_btab = nullptr;    // damping profile at half-cell distances (FP32 TMA passes)
    int nbtab = 0;
    double* d_kry = nullptr;
    long long* d_clk = nullptr;
    double* d_tclk = nullptr;
    long long version = 0;
    std::string err;
    long long launches = 0;
    struct Engine* engine = nullptr;
};

struct Engine {
    std::vector<ewv_model*> models;
    std::vector<long long> versions;
    std::vector<ProblemDev> probs;
    int nprob = 0, ntiles = 0, precision = 0, R = 4, dims = 2;
    int store_bf16 = 0;         // any model of the engine asked for bfloat16 storage rounding
    ProblemDev* d_probs = nullptr;
    int* d_tile_prob = nullptr;
    double* d_partials = nullptr;
    unsigned int* d_counters = nullptr;
    double* d_coef = nullptr;
    ProblemDev* d_apply = nullptr;
    void* d_maps = nullptr;     // FP32: TMA tensor maps of every problem
    int* d_tbase = nullptr;     // per 2D map set (TMA_SET_HEIGHTS): nprob + 1 tile prefix sums
    int* d_pbase = nullptr;     // nprob + 1 prefix sums of the flat pointwise chunks
    int nchunks = 0;
    int ntiles_by[TMA_NUM_SETS] = {};
    int tma_variant = -1;       // -1: choose by timing at first use
    double tma_variant_us[TMA_NUM_VARIANTS] = {};
    ProblemDev* d_adj = nullptr;  // adjoint call: descriptors (state = cotangent) + tile map
    void* d_adj_maps = nullptr;   // FP32: TMA tensor maps of the adjoint's buffers
    const void* adj_key_state = nullptr;     // ... valid for this cotangent buffer,
    const void* adj_key_work = nullptr;      // workspace
    size_t adj_key_bytes = 0;                // and workspace size
    std::vector<const void*> adj_tmaps;      // per-shot map pointers
    size_t d_adj_bytes = 0;
    ProblemDev* d_kadj = nullptr; // Krylov adjoint: three descriptor views of the workspace
    size_t d_kadj_bytes = 0;
    void* d_kexp_maps = nullptr;  // FP32 exponential Krylov adjoint: tensor maps of the
    const void* kexp_key_state = nullptr;    // forward and adjoint Arnoldi views, valid for
    const void* kexp_key_work = nullptr;     // this cotangent buffer, workspace,
    size_t kexp_key_bytes = 0;               // workspace size
    int kexp_key_m = 0;                      // and Krylov dimension
    std::vector<const void*> kexp_tmaps;     // per-view map pointers (2 nshots)
    double* d_kbar = nullptr;     // exact Krylov adjoint: per-shot reverse-sweep scalars
    size_t d_kbar_n = 0;
    // Krylov step with dense output (ewv_step_krylov_dense): the caller's buffer of the
    // four Gauss-Legendre states, set for the duration of that call only
    void* kry_dense = nullptr;
    // Gram-Schmidt column kernel: chunks per block for a co-resident grid (0: flat passes
    // only), double-buffered partials and the grid-barrier words
    int mgs_cpb = 0;
    double* d_mgs_partials = nullptr;
    unsigned int* d_mgs_bar = nullptr;
    double* d_ecoef = nullptr;    // [nprob][MAX_TAU][MAX_M]: exp(tau H) e_1 of a multi-output combine
    // adaptive Krylov step: tolerance, dimension range and statistics of the current call
    double ad_tol = 0.0;
    int ad_mmin = 1, ad_mmax = 1;
    int ad_stats[3] = {0, 0, 0};
    int* d_err = nullptr;       // error word: 1 = a bounded wait timed out (TMA pipeline or the
                                // Gram-Schmidt grid barrier), 2 = non-finite
    int* h_err = nullptr;       // pinned host copy, written by an async copy at the end of a call
    cudaEvent_t err_ev = nullptr;   // recorded after that copy
    std::map<std::tuple<double, int, double, double, double>, std::vector<double>> faber_cache;
    // CUDA graphs of one step's launch sequence, keyed by (method, m, dt, g, c0, c1, parity
    // + 2 x timing); a graph captured with timing on owns the event pairs around its passes
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        long long nodes = 0;
        std::vector<cudaEvent_t> ev;
        bool pending = false;   // launched with timing; event pairs not read yet
    };
    std::map<std::tuple<int, int, double, double, double, double, int>, StepGraph> graphs;
    bool graphs_enabled = true;
    bool graphs_broken = false;
    cudaStream_t cap = nullptr;              // capturable stream used while graphs are on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    void drop_graphs() {
        for (auto& kv : graphs) {
            StepGraph& sg = kv.second;
            if (sg.pending && cudaEventSynchronize(sg.ev.back()) == cudaSuccess) {
                for (size_t k = 0; k + 1 < sg.ev.size(); k += 2) {
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, sg.ev[k], sg.ev[k + 1]) == cudaSuccess) {
                        timing_acc_ms += ms;
                        ++timing_acc_n;
                    }
                }
            }
            cudaGraphExecDestroy(kv.second.exec);
            for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
        }
        graphs.clear();
    }
    // optional CUDA-event timing of the fused stencil passes (pairs around each launch);
    // replayed graphs add their pairs' times to timing_acc_* when they are read back
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    double timing_acc_ms = 0.0;
    long long timing_acc_n = 0;
    ~Engine() {
        if (err_ev) cudaEventSynchronize(err_ev);   // the last copy into h_err has landed
        drop_graphs();
        if (cap) cudaStreamDestroy(cap);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        cudaFree(d_probs);
        cudaFree(d_tile_prob);
        cudaFree(d_partials);
        cudaFree(d_counters);
        cudaFree(d_coef);
        cudaFree(d_apply);
        cudaFree(d_maps);
        cudaFree(d_tbase);
        cudaFree(d_pbase);
        cudaFree(d_err);
        if (h_err) cudaFreeHost(h_err);
        if (err_ev) cudaEventDestroy(err_ev);
        cudaFree(d_adj);
        cudaFree(d_adj_maps);
        cudaFree(d_kadj);
        cudaFree(d_kexp_maps);
        cudaFree(d_mgs_partials);
        cudaFree(d_mgs_bar);
        cudaFree(d_ecoef);
        cudaFree(d_kbar);
    }
};

struct ewv_batch {
    std::vector<ewv_model*> models;
    cudaStream_t stream = nullptr;
    bool stream_set = false;
    Engine* engine = nullptr;
    std::string err;
};

namespace {

// Krylov steps run each Arnoldi column's Gram-Schmidt steps on the column kernel when the
// engine's chunks fit one co-resident grid (ewv_debug_set_column_kernel(0) keeps the flat
// passes, for comparisons)
bool g_mgs_enabled = true;

// One column's Gram-Schmidt steps (first dot, then k = k0 .. kmax) on the column kernel over
// nprob problems laid out like the engine's (its chunk table); false if it cannot run.
bool mgs_column(Engine* E, int precision, const ProblemDev* probs, int nprob, int j, int k0, int kmax, int m,
                double tol, cudaStream_t s);

int fail(std::string& err, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return code;
}

#define CUDA_OR_FAIL(err, call)                                                              \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(err, EWV_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

bool aligned(const void* p) { return ((uintptr_t)p & 255u) == 0; }

// Extents (x, y, z) of field f: u, v (and psi in 3D) on the nodes; w_x, w_y, w_z one shorter
// along their axis.
void field_extent(const ewv_model* m, int f, int* ex, int* ey, int* ez) {
    *ex = m->d.nx - (f == 2 ? 1 : 0);
    *ey = m->d.ny - (f == 3 ? 1 : 0);
    *ez = m->nz - (f == 4 ? 1 : 0);
}

size_t compact_n(const ewv_model* m) {
    size_t n = 0;
    for (int f = 0; f < m->nfields; ++f) {
        int ex, ey, ez;
        field_extent(m, f, &ex, &ey, &ez);
        n += (size_t)ex * ey * ez;
    }
    return n;
}

void default_ellipse(const ewv_model* m, double* g, double* c0, double* c1) {
    const double kappa = m->d.free_surface ? 1.30 : 1.05;
    const double dims = (double)m->d.dims;
    const double omega = kappa * m->c_max * std::sqrt(dims * std::fabs(symbol_min(m->d.fd_order))) / m->d.dx;
    const double bsum = dims * m->d.beta0;
    const double ar = std::sqrt(2.0) * 0.5 * bsum;
    const double ai = std::sqrt(2.0) * omega;
    const double centre = -0.5 * bsum;
    *g = 0.5 * (ar + ai);
    *c0 = centre / *g;
    *c1 = (ar - ai) / (ar + ai);
}

void ellipse_of(const ewv_model* m, double* g, double* c0, double* c1) {
    if (m->ellipse_override) {
        *g = m->eg;
        *c0 = m->ec0;
        *c1 = m->ec1;
    } else {
        default_ellipse(m, g, c0, c1);
    }
}

int vectors_needed(int method, int m) {
    switch (method) {
        case EWV_METHOD_APPLY: return 0;
        case EWV_METHOD_FABER: return 2;
        case EWV_METHOD_KRYLOV: return m;
        case EWV_METHOD_HORK: return 2;
        case EWV_METHOD_RK32: return 2;
        case EWV_METHOD_RK44: return 3;
        case EWV_METHOD_LEAPFROG: return 1;
        case EWV_METHOD_ADJOINT_FABER: return m + 3;   // tape p_0..p_{m-1} + 3 cotangents
        case EWV_METHOD_ADJOINT_KRYLOV: return 2 * m + 9;  // two bases + 8 dense outputs
        case EWV_METHOD_ADJOINT_LEAPFROG: return 3;        // level-n tape, q, H^T q
        case EWV_METHOD_KRYLOV_ADAPTIVE: return m + 1;     // m = m_max: slots up to m_max + 2
        default: return -1;
    }
}

ProblemDev make_problem(ewv_model* m, int shot, int tile_base) {
    ProblemDev P{};
    const ewv_model_desc& d = m->d;
    P.nx = d.nx;
    P.ny = d.ny;
    P.pitch = m->pitch;
    P.fs = d.free_surface;
    P.pml = d.pml_width;
    P.nz = m->nz;
    P.nfields = m->nfields;
    P.tiles_x = (d.nx + BX - 1) / BX;
    P.tiles_y = (d.ny + BY - 1) / BY;
    P.tiles_z = m->nz > 1 ? (m->nz + KC3 - 1) / KC3 : 1;
    P.ntiles = P.tiles_x * P.tiles_y * P.tiles_z;
    P.tile_base = tile_base;
    const Shot& s = m->shots[shot];
    P.src_k = s.has_src ? s.sk : -1;
    P.shot = shot;
    P.has_src = s.has_src ? 1 : 0;
    P.src_i = s.has_src ? s.si : -1;
    P.src_j = s.has_src ? s.sj : -1;
    P.f_peak = s.f_peak;
    P.t0 = s.t0;
    P.amp = s.amp;
    P.nrec = (int)s.rec_off.size();
    P.rec_stride = d.max_receivers;
    P.capacity = m->seismo ? m->capacity : 0;
    P.p = d.src_taylor_p;
    P.beta0 = d.beta0;
    P.inv_dx = 1.0 / d.dx;
    P.inv_dx2 = 1.0 / (d.dx * d.dx);
    P.inv_pml = d.pml_width > 0 ? 1.0 / d.pml_width : 0.0;
    P.fbeta0 = (float)P.beta0;
    P.btab = m->d_btab;
    P.nbtab = m->nbtab;
    P.finv_pml = (float)P.inv_pml;
    P.finv_dx = (float)P.inv_dx;
    P.finv_dx2 = (float)P.inv_dx2;
    P.field_stride = (long long)m->field_elems;
    P.vec_stride = (long long)m->vec_elems;
    P.state = (char*)m->state + (size_t)shot * m->vec_elems * m->elem;
    P.work = m->work;
    P.c2 = m->params;
    P.sigma = m->d_sigma + (size_t)shot * MAX_SIGMA;
    P.rec_off = m->d_rec + (size_t)shot * (d.max_receivers > 0 ? d.max_receivers : 1);
    P.seismo = m->seismo ? (char*)m->seismo + (size_t)shot * m->capacity * d.max_receivers * m->elem
                         : nullptr;
    P.kry = m->d_kry + (size_t)shot * KRY_STRIDE;
    P.clk = m->d_clk + (size_t)shot * 4;
    P.tclk = m->d_tclk + (size_t)shot * 2;
    return P;
}

// Workspace per shot: `nvec` vectors; shots' workspaces are laid out back to back with a
// per-shot stride of (work_bytes / nshots) rounded down to whole vectors.
int build_engine(Engine* E, std::string& err) {
    E->drop_graphs();
    E->probs.clear();
    E->dims = E->models.empty() ? 2 : E->models[0]->d.dims;
    E->store_bf16 = 0;
    for (ewv_model* m : E->models) E->store_bf16 |= m->store_bf16;
    for (ewv_model* m : E->models)
        if (m->d.dims != E->dims) return fail(err, EWV_ERR_UNSUPPORTED, "a batch cannot mix 2D and 3D models");
    std::vector<int> work_vecs;
    int tb = 0;
    for (ewv_model* m : E->models) {
        const size_t per_shot = m->work ? (m->work_bytes / m->d.nshots) / (m->vec_elems * m->elem) : 0;
        for (int s = 0; s < m->d.nshots; ++s) {
            ProblemDev P = make_problem(m, s, tb);
            P.work = (m->work && per_shot > 0)
                         ? (char*)m->work + (size_t)s * per_shot * m->vec_elems * m->elem
                         : nullptr;
            tb += P.ntiles;
            E->probs.push_back(P);
            work_vecs.push_back((int)per_shot);
        }
    }
    E->nprob = (int)E->probs.size();
    E->ntiles = tb;
    {
        // flat pointwise passes: PCHUNK elements of a problem's padded vector per block
        std::vector<int> pb((size_t)E->nprob + 1, 0);
        int acc = 0;
        for (int p = 0; p < E->nprob; ++p) {
            ProblemDev& P = E->probs[p];
            const long long nel = (long long)P.nfields * P.field_stride;
            P.pchunks = (int)((nel + PCHUNK - 1) / PCHUNK);
            P.pchunk_base = acc;
            pb[p] = acc;
            acc += P.pchunks;
        }
        pb[E->nprob] = acc;
        E->nchunks = acc;
        // per-block (problem, chunk) pairs: a block finds its problem with one load
        pb.resize((size_t)flat_block_table(E->nprob) + 2 * (size_t)acc, 0);
        for (int p = 0, b = 0; p < E->nprob; ++p)
            for (int c = 0; c < E->probs[p].pchunks; ++c, ++b) {
                pb[(size_t)flat_block_table(E->nprob) + 2 * (size_t)b] = p;
                pb[(size_t)flat_block_table(E->nprob) + 2 * (size_t)b + 1] = c;
            }
        cudaFree(E->d_pbase);
        E->d_pbase = nullptr;
        CUDA_OR_FAIL(err, cudaMalloc(&E->d_pbase, sizeof(int) * pb.size()));
        CUDA_OR_FAIL(err, cudaMemcpy(E->d_pbase, pb.data(), sizeof(int) * pb.size(), cudaMemcpyHostToDevice));
        // the Gram-Schmidt column kernel, where every chunk fits one co-resident grid
        cudaFree(E->d_mgs_partials);
        cudaFree(E->d_mgs_bar);
        E->d_mgs_partials = nullptr;
        E->d_mgs_bar = nullptr;
        E->mgs_cpb = mgs_column_chunks_per_block(E->precision, E->nchunks);
        cudaFree(E->d_ecoef);
        E->d_ecoef = nullptr;
        CUDA_OR_FAIL(err, cudaMalloc(&E->d_ecoef, sizeof(double) * (size_t)E->nprob * MAX_TAU * MAX_M));
        if (E->mgs_cpb > 0) {
            CUDA_OR_FAIL(err, cudaMalloc(&E->d_mgs_partials, sizeof(double) * 2 * (size_t)E->nchunks));
            CUDA_OR_FAIL(err, cudaMalloc(&E->d_mgs_bar, sizeof(unsigned int) * 2));
            CUDA_OR_FAIL(err, cudaMemset(E->d_mgs_bar, 0, sizeof(unsigned int) * 2));
        }
    }
    if (E->precision == EWV_F32 && E->dims == 2) {
        if (build_tensor_maps(E->probs, E->R, work_vecs, &E->d_maps) != 0)
            return fail(err, EWV_ERR_CUDA, "TMA tensor-map encoding failed");
        std::vector<int> pre(TMA_NUM_SETS * (size_t)(E->nprob + 1), 0);
        const int* heights = TMA_SET_HEIGHTS;
        for (int set = 0; set < TMA_NUM_SETS; ++set) {
            int acc = 0;
            for (int p = 0; p < E->nprob; ++p) {
                pre[(size_t)set * (E->nprob + 1) + p] = acc;
                const ProblemDev& P = E->probs[p];
                acc += ((P.nx + BX - 1) / BX) * ((P.ny + heights[set] - 1) / heights[set]);
            }
            pre[(size_t)set * (E->nprob + 1) + E->nprob] = acc;
            E->ntiles_by[set] = acc;
        }
        cudaFree(E->d_tbase);
        E->d_tbase = nullptr;
        CUDA_OR_FAIL(err, cudaMalloc(&E->d_tbase, sizeof(int) * pre.size()));
        CUDA_OR_FAIL(err, cudaMemcpy(E->d_tbase, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice));
    }
    if (E->precision == EWV_F32 && E->dims == 3) {
        if (build_tensor_maps3d(E->probs, E->R, work_vecs, &E->d_maps) != 0)
            return fail(err, EWV_ERR_CUDA, "TMA tensor-map encoding failed (3D)");
        std::vector<int> pre((size_t)E->nprob + 1, 0);
        int acc = 0;
        for (int p = 0; p < E->nprob; ++p) {
            pre[p] = acc;
            acc += tma3d_tasks_of(E->probs[p]);
        }
        pre[E->nprob] = acc;
        E->ntiles_by[0] = acc;
        cudaFree(E->d_tbase);
        E->d_tbase = nullptr;
        CUDA_OR_FAIL(err, cudaMalloc(&E->d_tbase, sizeof(int) * pre.size()));
        CUDA_OR_FAIL(err, cudaMemcpy(E->d_tbase, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice));
    }
    if (!E->d_err) {
        CUDA_OR_FAIL(err, cudaMalloc(&E->d_err, sizeof(int)));
        CUDA_OR_FAIL(err, cudaMemset(E->d_err, 0, sizeof(int)));
        CUDA_OR_FAIL(err, cudaHostAlloc(&E->h_err, sizeof(int), cudaHostAllocDefault));
        *E->h_err = 0;
        CUDA_OR_FAIL(err, cudaEventCreateWithFlags(&E->err_ev, cudaEventDisableTiming));
    }
    std::vector<int> tp(tb);
    for (int p = 0; p < E->nprob; ++p)
        for (int t = 0; t < E->probs[p].ntiles; ++t) tp[E->probs[p].tile_base + t] = p;
    cudaFree(E->d_probs);
    cudaFree(E->d_tile_prob);
    cudaFree(E->d_partials);
    cudaFree(E->d_counters);
    E->d_probs = nullptr;
    E->d_tile_prob = nullptr;
    E->d_partials = nullptr;
    E->d_counters = nullptr;
    CUDA_OR_FAIL(err, cudaMalloc(&E->d_probs, sizeof(ProblemDev) * E->nprob));
    CUDA_OR_FAIL(err, cudaMalloc(&E->d_tile_prob, sizeof(int) * (size_t)tb));
    CUDA_OR_FAIL(err, cudaMalloc(&E->d_partials, sizeof(double) * (size_t)std::max(tb, E->nchunks)));
    CUDA_OR_FAIL(err, cudaMalloc(&E->d_counters, sizeof(unsigned int) * E->nprob));
    CUDA_OR_FAIL(err, cudaMemcpy(E->d_probs, E->probs.data(), sizeof(ProblemDev) * E->nprob,
                                 cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(err, cudaMemcpy(E->d_tile_prob, tp.data(), sizeof(int) * (size_t)tb,
                                 cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(err, cudaMemset(E->d_counters, 0, sizeof(unsigned int) * E->nprob));
    if (!E->d_coef) CUDA_OR_FAIL(err, cudaMalloc(&E->d_coef, sizeof(double) * (MAX_DEG + 1)));
    E->versions.clear();
    for (ewv_model* m : E->models) E->versions.push_back(m->version);
    return EWV_OK;
}

int engine_ready(Engine* E, std::string& err) {
    bool stale = E->probs.empty();
    for (size_t i = 0; i < E->models.size() && !stale; ++i)
        stale = E->versions[i] != E->models[i]->version;
    if (!stale) return EWV_OK;
    return build_engine(E, err);
}

int check_bound(ewv_model* m, int method, int mm, std::string& err) {
    if (!m->state || !m->params)
        return fail(err, EWV_ERR_NOT_BOUND, "state/params buffers are not bound");
    if (!m->velocity_set) return fail(err, EWV_ERR_NOT_BOUND, "velocity not set");
    const int nv = vectors_needed(method, mm);
    const size_t need = (size_t)nv * m->vec_elems * m->elem * m->d.nshots;
    if (m->work_bytes < need)
        return fail(err, EWV_ERR_WORKSPACE_TOO_SMALL, "workspace %zu bytes < %zu needed", m->work_bytes,
                    need);
    return EWV_OK;
}

StageArgs stage_defaults() {
    StageArgs a{};
    a.x = 0;
    a.u = a.a = a.y_out = a.acc_out = a.d = -1;
    a.src_slot = -1;
    a.x_scale_slot = -1;
    a.fin_mode = FIN_NONE;
    a.transpose = 0;
    return a;
}

// 3D engines: consumer warps of the TMA pass for the selected variant (2: 8 warps, else 16).
int tma3d_warps(const Engine* E) { return E->tma_variant == 2 ? 8 : 16; }

// Add the pass times of a timed graph's last replay (if not read yet) to the accumulator.
int harvest_graph_timing(Engine* E, Engine::StepGraph& sg, std::string& err) {
    if (!sg.pending) return EWV_OK;
    sg.pending = false;
    CUDA_OR_FAIL(err, cudaEventSynchronize(sg.ev.back()));
    for (size_t k = 0; k + 1 < sg.ev.size(); k += 2) {
        float ms = 0.f;
        CUDA_OR_FAIL(err, cudaEventElapsedTime(&ms, sg.ev[k], sg.ev[k + 1]));
        E->timing_acc_ms += ms;
        ++E->timing_acc_n;
    }
    return EWV_OK;
}

struct Ctx {
    Engine* E;
    cudaStream_t s;
    long long* launches;
    std::string* err;
    int launch_failed = 0;      // a TMA pass could not be configured or launched
    std::vector<cudaEvent_t>* capture_ev = nullptr;   // set while a timed step is captured
    cudaEvent_t next_event() {
        if (capture_ev) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            capture_ev->push_back(e);
            return e;
        }
        if (E->events_used == E->events.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            E->events.push_back(e);
        }
        return E->events[E->events_used++];
    }
    // Launch one stencil-type kernel through `launch` with the per-launch timing events that
    // stage() records (kernel timing on), and count it.
    template <class F>
    void timed(F&& launch) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        const unsigned rec_flags = capture_ev ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (E->timing) {
            e0 = next_event();
            e1 = next_event();
            cudaEventRecordWithFlags(e0, s, rec_flags);
        }
        launch();
        if (E->timing) cudaEventRecordWithFlags(e1, s, rec_flags);
        ++*launches;
    }
    void stage(const StageArgs& a_in) {
        StageArgs a = a_in;
        a.store_bf16 = E->store_bf16;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        const unsigned rec_flags = capture_ev ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (E->timing) {
            e0 = next_event();
            e1 = next_event();
            cudaEventRecordWithFlags(e0, s, rec_flags);
        }
        if (E->dims == 3) {
            // FP32 passes without a dot product take the TMA pipeline (variant 0: 16 consumer
            // warps, 2: 8 warps) unless variant 1 (the plain z-marching kernel) is selected
            if (a.transpose || a.grad) launch_failed = 1;   // 3D has no adjoint pass
            else if (E->precision == EWV_F32 && a.fin_mode == FIN_NONE && a.d < 0 && E->tma_variant != 1) {
                if (launch_stage_tma3d(E->R, tma3d_warps(E), E->d_probs, E->d_tbase, E->nprob,
                                       E->ntiles_by[0], a, E->d_err, s) != 0)
                    launch_failed = 1;
            } else {
                launch_stage3d(E->precision, E->R, E->ntiles, E->d_probs, E->d_tile_prob, a, s);
            }
        } else if (E->precision == EWV_F32 && a.transpose && a.fin_mode == FIN_NONE && a.d < 0 && !a.grad &&
                   !a.store_bf16 && E->d_tbase) {
            const int set = tma_map_set(18);
            if (launch_transpose_tma(E->R, E->d_probs, E->d_tbase + (size_t)set * (E->nprob + 1), E->nprob,
                                     E->ntiles_by[set], a, E->d_err, s) != 0)
                launch_failed = 1;
        } else if (E->precision == EWV_F32 && !a.transpose && a.fin_mode == FIN_NONE && a.d < 0 && !a.grad &&
                   !a.store_bf16) {
            if (E->tma_variant < 0) autotune();
            if (E->tma_variant < 0) {
                launch_failed = 1;
            } else {
                const int set = tma_map_set(tma_variant_tile_height_for(E->tma_variant, a.a >= 0));
                if (launch_stage_tma(E->tma_variant, E->R, E->d_probs, E->d_tbase + (size_t)set * (E->nprob + 1),
                                     E->nprob, E->ntiles_by[set], a, E->d_err, s) != 0)
                    launch_failed = 1;
            }
        } else
            launch_stage(E->precision, E->R, E->ntiles, E->d_probs, E->d_tile_prob, a, s);
        if (E->timing) cudaEventRecordWithFlags(e1, s, rec_flags);
        ++*launches;
    }
    void point(const PointArgs& pa) {
        if (pa.mode <= 2 || pa.mode == 5 || pa.mode == 7 || pa.mode == 8)   // norm, MGS, combines, dots: flat
            launch_point_flat(E->precision, E->nchunks, E->d_probs, E->d_pbase, E->nprob, pa, s);
        else
            launch_point(E->precision, E->ntiles, E->d_probs, E->d_tile_prob, pa, s);
        ++*launches;
    }
    // Tile-shape autotuner: time every persistent-kernel variant on two idempotent probe
    // passes (read the state, write workspace vectors 1 and 2, which every FP32 method
    // overwrites before reading): one with a U and an A operand (the Faber and low-storage
    // HORK form) and one with U only (the Horner HORK form); keep the variant with the
    // smallest sum.  Runs once per engine, outside graph capture.
    void autotune() {
        StageArgs p = stage_defaults();
        p.x = 0;
        p.u = 0;
        p.a = 0;
        p.y_out = 1;
        p.acc_out = 2;
        p.cx = 1.0;
        p.ch = 1e-3;
        p.cu = 1.0;
        p.ck = 1.0;
        p.ca = 1.0;
        p.cay = 1.0;
        StageArgs pn = p;           // no A operand, no accumulator
        pn.a = -1;
        pn.acc_out = -1;
        pn.ca = 0.0;
        pn.cay = 0.0;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        int best = -1;
        double best_us = 1e300;
        for (int v = 0; v < TMA_NUM_VARIANTS; ++v) {
            const int set = tma_map_set(tma_variant_tile_height_for(v, true));
            const int setn = tma_map_set(tma_variant_tile_height_for(v, false));
            const int* tb = E->d_tbase + (size_t)set * (E->nprob + 1);
            const int* tbn = E->d_tbase + (size_t)setn * (E->nprob + 1);
            if (launch_stage_tma(v, E->R, E->d_probs, tb, E->nprob, E->ntiles_by[set], p, E->d_err, s) != 0 ||
                launch_stage_tma(v, E->R, E->d_probs, tbn, E->nprob, E->ntiles_by[setn], pn, E->d_err, s) != 0 ||
                cudaGetLastError() != cudaSuccess) {
                E->tma_variant_us[v] = -1.0;
                continue;
            }
            double best_v = 1e300;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                launch_stage_tma(v, E->R, E->d_probs, tb, E->nprob, E->ntiles_by[set], p, E->d_err, s);
                launch_stage_tma(v, E->R, E->d_probs, tbn, E->nprob, E->ntiles_by[setn], pn, E->d_err, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best_v = std::min(best_v, 1e3 * (double)ms);
            }
            // a variant whose pipeline wait gave up is not a candidate (clear its flag)
            int flag = 0;
            if (cudaMemcpyAsync(&flag, E->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess || flag != 0) {
                cudaMemsetAsync(E->d_err, 0, sizeof(int), s);
                E->tma_variant_us[v] = -1.0;
                continue;
            }
            E->tma_variant_us[v] = best_v;
            if (best_v < best_us) {
                best_us = best_v;
                best = v;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        E->tma_variant = best;
        *launches += 8 * TMA_NUM_VARIANTS;
    }
    void copy(int src, int dst, int fmask, bool swap) {
        PointArgs pa{};
        pa.mode = swap ? 4 : 3;
        pa.src = src;
        pa.dst = dst;
        pa.fmask = fmask;
        point(pa);
    }
    void prologue(int kind, int m, double g = 0, double c0 = 0, double c1 = 0) {
        launch_prologue(E->d_probs, E->nprob, kind, m, g, c0, c1, s);
        ++*launches;
    }
    void record(int vec = 0) {
        launch_record(E->precision, E->d_probs, E->nprob, vec, s);
        ++*launches;
    }
    // Run nsteps steps.  Steps are parameter-free (time comes from the device clock), so
    // after the first step(s) the launch sequence of one step is captured once into a CUDA
    // graph and replayed; `nparity` distinct sequences alternate (leap-frog buffer swap).
    // With kernel timing on, the captured step records its own event pairs (external event
    // nodes); two copies of each graph alternate, and a copy's pairs are read back just
    // before its next replay, while the other copy keeps the GPU busy.  A failed capture
    // falls back to direct launches for this engine.
    template <class F>
    int step_loop(int nsteps, int method, int m, double dt, double g, double c0, double c1,
                  int nparity, F&& one_step) {
        for (int n = 0; n < nsteps; ++n) {
            const int par = n % nparity;
            const int slot = E->timing ? 2 + 2 * ((n / nparity) & 1) : 0;
            auto key = std::make_tuple(method, m, dt, g, c0, c1, par + slot);
            // the first steps of a call launch directly (one-time work such as the tile-shape
            // tuning happens there), unless an earlier call already captured this step
            const bool ok = E->graphs_enabled && !E->graphs_broken;
            auto it = ok ? E->graphs.find(key) : E->graphs.end();
            if (!ok || (n < nparity && it == E->graphs.end())) {
                one_step(n);
                continue;
            }
            if (it == E->graphs.end()) {
                const long long L0 = *launches;
                Engine::StepGraph sg;
                cudaGraph_t gr = nullptr;
                if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    cudaGetLastError();
                    E->graphs_broken = true;
                    one_step(n);
                    continue;
                }
                if (E->timing) capture_ev = &sg.ev;
                one_step(n);
                capture_ev = nullptr;
                const cudaError_t e1 = cudaStreamEndCapture(s, &gr);
                sg.nodes = *launches - L0;
                *launches = L0;
                if (e1 != cudaSuccess || cudaGraphInstantiate(&sg.exec, gr, 0) != cudaSuccess) {
                    if (gr) cudaGraphDestroy(gr);
                    for (cudaEvent_t ev : sg.ev) cudaEventDestroy(ev);
                    cudaGetLastError();
                    E->graphs_broken = true;
                    one_step(n);
                    continue;
                }
                cudaGraphDestroy(gr);
                it = E->graphs.emplace(key, std::move(sg)).first;
            }
            Engine::StepGraph& sg = it->second;
            if (harvest_graph_timing(E, sg, *err) != EWV_OK) return EWV_ERR_CUDA;
            const cudaError_t e = cudaGraphLaunch(sg.exec, s);
            if (e != cudaSuccess) return fail(*err, EWV_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
            *launches += sg.nodes;
            sg.pending = !sg.ev.empty();
        }
        return EWV_OK;
    }
};

int check_launch(std::string& err) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(err, EWV_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return EWV_OK;
}

// ---------------------------------------------------------------- step plans
int run_faber(Ctx& C, double t, double dt, int m, int nsteps, double g, double c0, double c1) {
    std::string& err = *C.err;
    if (m < 1 || m > MAX_DEG) return fail(err, EWV_ERR_INVALID_ARG, "Faber degree must be 1..%d", MAX_DEG);
    auto key = std::make_tuple(dt, m, g, c0, c1);
    auto it = C.E->faber_cache.find(key);
    if (it == C.E->faber_cache.end()) {
        launch_faber_coeffs(dt, g, c0, c1, m, C.E->d_coef, C.s);
        ++*C.launches;
        std::vector<double> a(m + 1);
        CUDA_OR_FAIL(err, cudaMemcpyAsync(a.data(), C.E->d_coef, sizeof(double) * (m + 1),
                                          cudaMemcpyDeviceToHost, C.s));
        CUDA_OR_FAIL(err, cudaStreamSynchronize(C.s));
        it = C.E->faber_cache.emplace(key, a).first;
    }
    const std::vector<double>& a = it->second;
    launch_set_clock(C.E->d_probs, C.E->nprob, t, dt, C.s);
    ++*C.launches;
    int rc = C.step_loop(nsteps, EWV_METHOD_FABER, m, dt, g, c0, c1, 1, [&](int) {
        C.prologue(PRO_FABER, m, g, c0, c1);
        StageArgs s1 = stage_defaults();
        s1.x = 0;
        s1.y_out = 1;
        s1.acc_out = 2;
        s1.src_slot = 0;
        s1.cx = -c0;
        s1.ch = 1.0 / g;
        s1.ck = 1.0;
        s1.cay = a[1];
        s1.cax = a[0];
        C.stage(s1);
        if (m == 1) {
            C.copy(2, 0, ALL_FIELDS, false);
        } else {
            StageArgs s2 = stage_defaults();
            s2.x = 1;
            s2.u = 0;
            s2.a = 2;
            s2.y_out = 2;
            s2.acc_out = 0;
            s2.src_slot = 1;
            s2.cx = -c0;
            s2.ch = 1.0 / g;
            s2.cu = -2.0 * c1;
            s2.ck = 1.0;
            s2.ca = 1.0;
            s2.cay = a[2];
            C.stage(s2);
            for (int j = 3; j <= m; ++j) {
                StageArgs sj = stage_defaults();
                const int in = (j & 1) ? 2 : 1;
                const int out = (j & 1) ? 1 : 2;
                sj.x = in;
                sj.u = out;
                sj.a = 0;
                sj.y_out = out;
                sj.acc_out = 0;
                sj.src_slot = j - 1;
                sj.cx = -c0;
                sj.ch = 1.0 / g;
                sj.cu = -c1;
                sj.ck = 1.0;
                sj.ca = 1.0;
                sj.cay = a[j];
                C.stage(sj);
            }
        }
        C.record();
    });
    if (rc != EWV_OK) return rc;
    return check_launch(err);
}

std::vector<double> hork_lambdas(int m) {
    // lambda^(1) = [1]; lambda^(q)_k = lambda^(q-1)_{k-1}/k (k = 1..q-2),
    // lambda^(q)_{q-1} = 1/q!, lambda^(q)_0 = 1 - sum of the others.
    std::vector<double> lam(1, 1.0);
    double fact = 1.0;
    for (int q = 2; q <= m; ++q) {
        fact *= q;
        std::vector<double> nl(q, 0.0);
        for (int k = 1; k <= q - 2; ++k) nl[k] = lam[k - 1] / k;
        nl[q - 1] = 1.0 / fact;
        double s = 0.0;
        for (int k = 1; k < q; ++k) s += nl[k];
        nl[0] = 1.0 - s;
        lam = nl;
    }
    return lam;
}

// HORK(m) in Horner form: the same degree-m Taylor polynomial of exp(dt H~) as the
// low-storage stages below, evaluated as V_{m+1} = V_0, V_j = V_0 + (dt/j) H~ V_{j+1}
// (j = m .. 1), U^{n+1} = V_1.  Each pass reads V_{j+1} (with halo), V_0 and c^2 and writes
// V_j: 13 words per point against 17 for a stage with an accumulator.  Rounding made in
// pass j reaches the result multiplied by (dt H~)^(j-1)/(j-1)!, which is large on the top of
// the spectrum at large steps.  Work vectors 1 and 2 alternate; the last pass writes the
// state in place (V_0 is read only at the point being written).
int run_hork_horner(Ctx& C, double t, double dt, int m, int nsteps) {
    launch_set_clock(C.E->d_probs, C.E->nprob, t, dt, C.s);
    ++*C.launches;
    int rc = C.step_loop(nsteps, EWV_METHOD_HORK, m, dt, 0, 0, 0, 1, [&](int) {
        C.prologue(PRO_HORK_HORNER, m);
        int prev = 0;
        for (int k = 0; k < m; ++k) {
            const int j = m - k;
            StageArgs s = stage_defaults();
            s.x = prev;
            s.src_slot = k;
            s.ch = dt / (double)j;
            s.ck = 1.0;
            if (k == 0) {
                s.cx = 1.0;                     // V_m = V_0 + (dt/m) H~ V_0
            } else {
                s.cx = 0.0;
                s.u = 0;
                s.cu = 1.0;
            }
            s.y_out = (j == 1 && k > 0) ? 0 : (prev == 1 ? 2 : 1);
            C.stage(s);
            prev = s.y_out;
        }
        if (prev != 0) C.copy(prev, 0, ALL_FIELDS, false);   // m = 1: V_1 is in a work vector
        C.record();
    });
    if (rc != EWV_OK) return rc;
    return check_launch(*C.err);
}

int run_hork(Ctx& C, double t, double dt, int m, int nsteps) {
    std::string& err = *C.err;
    if (m < 1 || m > MAX_SIGMA) return fail(err, EWV_ERR_INVALID_ARG, "HORK stages must be 1..%d", MAX_SIGMA);
    if (!C.E->models.empty() && C.E->models[0]->hork_form == EWV_HORK_HORNER)
        return run_hork_horner(C, t, dt, m, nsteps);
    const std::vector<double> lam = hork_lambdas(m);
    auto wgt = [&](int i) { return i <= m - 2 ? lam[i] : (i == m - 1 ? 0.0 : lam[m - 1]); };
    launch_set_clock(C.E->d_probs, C.E->nprob, t, dt, C.s);
    ++*C.launches;
    int rc = C.step_loop(nsteps, EWV_METHOD_HORK, m, dt, 0, 0, 0, 1, [&](int) {
        C.prologue(PRO_HORK, m);
        if (m == 1) {
            StageArgs s1 = stage_defaults();
            s1.x = 0;
            s1.acc_out = 1;
            s1.src_slot = 0;
            s1.cx = 1.0;
            s1.ch = dt;
            s1.ck = 1.0;
            s1.cay = lam[0];
            C.stage(s1);
            C.copy(1, 0, ALL_FIELDS, false);
            C.record();
            return;
        }
        for (int i = 1; i <= m; ++i) {
            StageArgs si = stage_defaults();
            si.cx = 1.0;
            si.ch = dt;
            si.ck = 1.0;
            si.src_slot = i - 1;
            if (i == 1) {
                si.x = 0;
                si.y_out = 1;
                si.acc_out = 2;
                si.cax = lam[0];
                si.cay = wgt(1);
            } else if (i == 2) {
                si.x = 1;
                si.y_out = (m > 2) ? 2 : -1;
                si.a = 2;
                si.acc_out = 0;
                si.ca = 1.0;
                si.cay = wgt(2);
            } else {
                si.x = ((i - 1) & 1) ? 1 : 2;
                si.y_out = (i < m) ? ((i & 1) ? 1 : 2) : -1;
                si.a = 0;
                si.acc_out = 0;
                si.ca = 1.0;
                si.cay = wgt(i);
            }
            C.stage(si);
        }
        C.record();
    });
    if (rc != EWV_OK) return rc;
    return check_launch(err);
}

int run_rk(Ctx& C, double t, double dt, int scheme, int nsteps) {
    launch_set_clock(C.E->d_probs, C.E->nprob, t, dt, C.s);
    ++*C.launches;
    int rc = C.step_loop(nsteps, scheme, 0, dt, 0, 0, 0, 1, [&](int) {
        if (scheme == EWV_METHOD_RK32) {
            C.prologue(PRO_RK32, 3);
            const int xs[3] = {0, 1, 2}, ys[3] = {1, 2, 0};
            const double al[3] = {0.5 * dt, 0.5 * dt, dt};
            for (int q = 0; q < 3; ++q) {
                StageArgs a = stage_defaults();
                a.x = xs[q];
                a.u = 0;
                a.y_out = ys[q];
                a.src_slot = q;
                a.ch = 1.0;
                a.cu = 1.0;
                a.ck = al[q];
                C.stage(a);
            }
        } else {
            C.prologue(PRO_RK44, 4);
            StageArgs a = stage_defaults();
            a.x = 0; a.u = 0; a.y_out = 1; a.acc_out = 3; a.src_slot = 0;
            a.ch = 1.0; a.cu = 1.0; a.ck = 0.5 * dt; a.cau = 1.0; a.cak = dt / 6.0;
            C.stage(a);
            a = stage_defaults();
            a.x = 1; a.u = 0; a.a = 3; a.y_out = 2; a.acc_out = 3; a.src_slot = 1;
            a.ch = 1.0; a.cu = 1.0; a.ck = 0.5 * dt; a.ca = 1.0; a.cak = dt / 3.0;
            C.stage(a);
            a = stage_defaults();
            a.x = 2; a.u = 0; a.a = 3; a.y_out = 1; a.acc_out = 3; a.src_slot = 2;
            a.ch = 1.0; a.cu = 1.0; a.ck = dt; a.ca = 1.0; a.cak = dt / 3.0;
            C.stage(a);
            a = stage_defaults();
            a.x = 1; a.a = 3; a.acc_out = 0; a.src_slot = 3;
            a.ch = 1.0; a.ca = 1.0; a.cak = dt / 6.0;
            C.stage(a);
        }
        C.record();
    });
    if (rc != EWV_OK) return rc;
    return check_launch(*C.err);
}

bool mgs_column(Engine* E, int precision, const ProblemDev* probs, int nprob, int j, int k0, int kmax, int m,
                double tol, cudaStream_t s) {
    if (E->mgs_cpb <= 0 || nprob != E->nprob || !E->d_mgs_partials || !E->d_mgs_bar) return false;
    MgsArgs ma{};
    ma.j = j;
    ma.k0 = k0;
    ma.kmax = kmax;
    ma.m = m;
    ma.tol = tol;
    ma.partials = E->d_mgs_partials;
    ma.bar = E->d_mgs_bar;
    ma.err = E->d_err;
    return launch_mgs_column(precision, E->nchunks, E->mgs_cpb, probs, E->d_pbase, nprob, ma, s) == 0;
}

int run_krylov(Ctx& C, double t, double dt, int m, int nsteps, int* info) {
    std::string& err = *C.err;
    if (m < 1 || m > MAX_M) return fail(err, EWV_ERR_INVALID_ARG, "Krylov m must be 1..%d", MAX_M);
    const double tol = C.E->precision == EWV_F64 ? 1e-14 : 1e-6;
    launch_set_clock(C.E->d_probs, C.E->nprob, t, dt, C.s);
    ++*C.launches;
    bool expm_ok = true;
    const int window = C.E->models.empty() ? 0 : C.E->models[0]->kry_window;
    // FP32: the matrix-vector product runs on the TMA stencil pass, which has no dot partner;
    // a flat pass then forms <q_{j+1}, q_k0> with the same finalisation (FP64 keeps the fused
    // dot of the plain stencil kernel)
    const bool split_dot = C.E->precision == EWV_F32;
    // dense output: before the step's own combine (which overwrites q_1 = U^{n-1}), the states
    // x(tau_q dt) = beta V exp(tau_q H_m) e_1 at the 4-point Gauss-Legendre nodes go to the
    // caller's buffer [q][shot]; a key of its own keeps such a call out of the step graphs
    void* const dense = C.E->kry_dense;
    static const double kTauGL[4] = {0.069431844202973712, 0.33000947820757187,
                                     0.66999052179242813, 0.93056815579702629};
    const long long vel = C.E->nprob > 0 ? (long long)C.E->models[0]->vec_elems : 0;
    const int key_method = dense ? -EWV_METHOD_KRYLOV : EWV_METHOD_KRYLOV;
    int rc0 = C.step_loop(nsteps, key_method, m, dt, tol, (double)window, 0, 1, [&](int) {
        C.prologue(PRO_KRYLOV, m);
        PointArgs pn{};
        pn.mode = 0;
        pn.m = m;
        pn.tol = tol;
        pn.partials = C.E->d_partials;
        pn.counters = C.E->d_counters;
        C.point(pn);
        const bool col = g_mgs_enabled && C.E->mgs_cpb > 0;
        for (int j = 1; j <= m; ++j) {
            // orthogonalise q_{j+1} against q_{k0} .. q_j (all of them without a window)
            const int k0 = window > 0 ? std::max(1, j - window + 1) : 1;
            StageArgs a = stage_defaults();
            a.x = j - 1;
            a.y_out = j;
            a.d = k0 - 1;
            a.src_slot = j;
            a.x_scale_slot = KRY_S + j;
            a.ch = dt;
            a.ck = 1.0;
            a.fin_mode = FIN_MATVEC;
            a.fin_j = j;
            a.fin_k = k0;
            a.m = m;
            a.tol = tol;
            a.partials = C.E->d_partials;
            a.counters = C.E->d_counters;
            if (split_dot || col) {
                a.d = -1;
                a.fin_mode = FIN_NONE;
            }
            C.stage(a);
            if (col && mgs_column(C.E, C.E->precision, C.E->d_probs, C.E->nprob, j, k0, (j == m) ? j - 1 : j, m,
                                  tol, C.s)) {
                ++*C.launches;
                continue;
            }
            if (split_dot || col) {        // (col: the column kernel could not be launched)
                PointArgs pd{};
                pd.mode = 5;
                pd.j = j;
                pd.k = k0;
                pd.m = m;
                pd.tol = tol;
                pd.partials = C.E->d_partials;
                pd.counters = C.E->d_counters;
                C.point(pd);
            }
            // at j = m the pass k = m only feeds h_{m+1,m}, which the result does not use
            const int kmax = (j == m) ? j - 1 : j;
            for (int k = k0; k <= kmax; ++k) {
                PointArgs pm{};
                pm.mode = 1;
                pm.j = j;
                pm.k = k;
                pm.m = m;
                pm.tol = tol;
                pm.partials = C.E->d_partials;
                pm.counters = C.E->d_counters;
                C.point(pm);
            }
        }
        if (dense) {
            // the four dense states and the step's result from one read of the basis
            const double taus[5] = {kTauGL[0], kTauGL[1], kTauGL[2], kTauGL[3], 1.0};
            if (launch_expm_multi(C.E->d_probs, C.E->nprob, m, C.s, taus, 5, C.E->d_ecoef) != 0) expm_ok = false;
            ++*C.launches;
            PointArgs pq{};
            pq.mode = 8;
            pq.m = m;
            pq.nout = 4;
            pq.final_out = 1;
            pq.ecoef = C.E->d_ecoef;
            pq.out = dense;
            pq.out_stride = vel;
            pq.out_qstride = (long long)C.E->nprob * vel;
            C.point(pq);
        } else {
            if (launch_expm(C.E->d_probs, C.E->nprob, m, C.s) != 0) expm_ok = false;
            ++*C.launches;
            PointArgs pc{};
            pc.mode = 2;
            pc.m = m;
            C.point(pc);
        }
        C.record();
    });
    if (rc0 != EWV_OK) return rc0;
    if (!expm_ok) return fail(err, EWV_ERR_CUDA, "expm shared-memory configuration failed");
    int rc = check_launch(err);
    if (rc != EWV_OK) return rc;
    // Without an info pointer the call does not wait: a non-finite Arnoldi value reaches the
    // host through the error word (the end-of-call scan reads the flag).  With one, read
    // back the effective dimensions and the non-finite flags now.
    if (!info) return EWV_OK;
    int meff_min = m;
    bool nonfinite = false;
    for (ewv_model* md : C.E->models) {
        std::vector<double> kb((size_t)md->d.nshots * KRY_STRIDE);
        CUDA_OR_FAIL(err, cudaMemcpyAsync(kb.data(), md->d_kry, kb.size() * sizeof(double),
                                          cudaMemcpyDeviceToHost, C.s));
        CUDA_OR_FAIL(err, cudaStreamSynchronize(C.s));
        for (int s = 0; s < md->d.nshots; ++s) {
            const double* k = kb.data() + (size_t)s * KRY_STRIDE;
            meff_min = std::min(meff_min, (int)k[KRY_MEFF]);
            if (k[KRY_NONFINITE] != 0.0) nonfinite = true;
        }
    }
    if (info) *info = meff_min;
    if (nonfinite) return fail(err, EWV_ERR_NONFINITE, "non-finite value in the Arnoldi process");
    return EWV_OK;
}

// exp(A) of a dense n x n matrix (row-major) by the [13/13] Pade approximant with scaling and
// squaring (Higham 2005), in FP64 on the host: the small dense part of the reverse sweep.
std::vector<double> host_expm(const std::vector<double>& A0, int n) {
    auto mul = [n](const std::vector<double>& X, const std::vector<double>& Y) {
        std::vector<double> Z((size_t)n * n, 0.0);
        for (int r = 0; r < n; ++r)
            for (int k = 0; k < n; ++k) {
                const double x = X[(size_t)r * n + k];
                if (x == 0.0) continue;
                for (int c = 0; c < n; ++c) Z[(size_t)r * n + c] += x * Y[(size_t)k * n + c];
            }
        return Z;
    };
    double f[27];
    f[0] = 1.0;
    for (int i = 1; i <= 26; ++i) f[i] = f[i - 1] * i;
    double b[14];
    for (int k = 0; k <= 13; ++k) b[k] = f[26 - k] * f[13] / (f[26] * f[k] * f[13 - k]);
    double nrm = 0.0;
    for (int c = 0; c < n; ++c) {
        double cs = 0.0;
        for (int r = 0; r < n; ++r) cs += std::fabs(A0[(size_t)r * n + c]);
        nrm = std::max(nrm, cs);
    }
    const double theta13 = 5.371920351148152;
    const int sc = nrm > theta13 ? (int)std::ceil(std::log2(nrm / theta13)) : 0;
    std::vector<double> A(A0);
    const double fac = std::ldexp(1.0, -sc);
    for (double& v : A) v *= fac;
    const std::vector<double> A2 = mul(A, A), A4 = mul(A2, A2), A6 = mul(A4, A2);
    const size_t nn = (size_t)n * n;
    std::vector<double> T1(nn), T2(nn);
    for (size_t e = 0; e < nn; ++e) T1[e] = b[13] * A6[e] + b[11] * A4[e] + b[9] * A2[e];
    std::vector<double> U = mul(A6, T1);
    for (size_t e = 0; e < nn; ++e) U[e] += b[7] * A6[e] + b[5] * A4[e] + b[3] * A2[e];
    for (int r = 0; r < n; ++r) U[(size_t)r * n + r] += b[1];
    U = mul(A, U);
    for (size_t e = 0; e < nn; ++e) T2[e] = b[12] * A6[e] + b[10] * A4[e] + b[8] * A2[e];
    std::vector<double> V = mul(A6, T2);
    for (size_t e = 0; e < nn; ++e) V[e] += b[6] * A6[e] + b[4] * A4[e] + b[2] * A2[e];
    for (int r = 0; r < n; ++r) V[(size_t)r * n + r] += b[0];
    // solve (V - U) X = (V + U) by Gaussian elimination with partial pivoting
    std::vector<double> L(nn), X(nn);
    for (size_t e = 0; e < nn; ++e) {
        L[e] = V[e] - U[e];
        X[e] = V[e] + U[e];
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(L[(size_t)r * n + c]) > std::fabs(L[(size_t)piv * n + c])) piv = r;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(L[(size_t)c * n + k], L[(size_t)piv * n + k]);
                std::swap(X[(size_t)c * n + k], X[(size_t)piv * n + k]);
            }
        const double d = L[(size_t)c * n + c];
        for (int r = c + 1; r < n; ++r) {
            const double fct = L[(size_t)r * n + c] / d;
            if (fct == 0.0) continue;
            for (int k = c; k < n; ++k) L[(size_t)r * n + k] -= fct * L[(size_t)c * n + k];
            for (int k = 0; k < n; ++k) X[(size_t)r * n + k] -= fct * X[(size_t)c * n + k];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        const double d = L[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            double v = X[(size_t)c * n + k];
            for (int q = c + 1; q < n; ++q) v -= L[(size_t)c * n + q] * X[(size_t)q * n + k];
            X[(size_t)c * n + k] = v / d;
        }
    }
    for (int i = 0; i < sc; ++i) X = mul(X, X);
    return X;
}


// (exp(tau H) e_1, tau phi_1(tau H) e_1, tau^2 phi_2(tau H) e_1) for the j x j Hessenberg H
// (row-major, stride MAX_M in kry) from one exponential of the twice-bordered matrix
// [[tau H, tau e_1, 0], [0, 0, tau], [0, 0, 0]].
void phi_block(const double* kry, int j, double tau, std::vector<double>& e, double& ph1_last,
               double& ph2_last) {
    const int n = j + 2;
    std::vector<double> B((size_t)n * n, 0.0);
    for (int r = 0; r < j; ++r)
        for (int c = 0; c < j; ++c) B[(size_t)r * n + c] = tau * kry[KRY_H + r * MAX_M + c];
    B[(size_t)0 * n + j] = tau;
    B[(size_t)j * n + j + 1] = tau;
    const std::vector<double> E = host_expm(B, n);
    e.assign(j, 0.0);
    for (int r = 0; r < j; ++r) e[r] = E[(size_t)r * n];
    ph1_last = E[(size_t)(j - 1) * n + j];
    ph2_last = E[(size_t)(j - 1) * n + j + 1];
}

// Adaptive Krylov step (KIOPS-style dimension and substep control; the paper names it as the
// improvement it leaves out, Secs. 3.2 and 6).  On the augmented A = dt H~_eta each substep
// grows the basis one vector at a time from m_min to m_max and stops at the first j whose
// two-term estimate beta h_{j+1,j} (tau |[phi_1(tau H_j)]_{j,1}| + tau^2 |[phi_2(tau H_j)]_{j,1}|
// |A v_{j+1}|) is at most tol tau beta; A v_{j+1} is the next column's matrix-vector product,
// computed once and reused.  At m_max without success tau shrinks on the same basis; after
// a substep tau grows by at most 2x.  A happy breakdown takes the rest of the step at once.
// Every problem has its own dimensions and substeps: the host reads the Krylov scalars after
// each column, decides, and marks finished problems inactive (KRY_ACTIVE, KRY_SKIP).
int run_krylov_adaptive(Ctx& C, double t, double dt, double tol, int mmin, int mmax, int nsteps,
                        int* stats) {
    std::string& err = *C.err;
    Engine* E = C.E;
    if (mmin < 1 || mmax < mmin || mmax + 1 > MAX_M || !(tol > 0.0))
        return fail(err, EWV_ERR_INVALID_ARG, "adaptive Krylov: need 1 <= m_min <= m_max <= %d, tol > 0", MAX_M - 1);
    const int np = E->nprob;
    const double btol = E->precision == EWV_F64 ? 1e-14 : 1e-6;
    const int window = E->models.empty() ? 0 : E->models[0]->kry_window;
    std::vector<std::vector<double>> kb((size_t)np, std::vector<double>(KRY_STRIDE));
    auto read_all = [&]() -> int {
        for (int p = 0; p < np; ++p)
            CUDA_OR_FAIL(err, cudaMemcpyAsync(kb[p].data(), E->probs[p].kry, sizeof(double) * KRY_STRIDE,
                                              cudaMemcpyDeviceToHost, C.s));
        CUDA_OR_FAIL(err, cudaStreamSynchronize(C.s));
        for (int p = 0; p < np; ++p)
            if (kb[p][KRY_NONFINITE] != 0.0)
                return fail(err, EWV_ERR_NONFINITE, "non-finite value in the Arnoldi process");
        return EWV_OK;
    };
    auto write = [&](int p) -> int {
        CUDA_OR_FAIL(err, cudaMemcpyAsync(E->probs[p].kry, kb[p].data(), sizeof(double) * KRY_STRIDE,
                                          cudaMemcpyHostToDevice, C.s));
        return EWV_OK;
    };
    auto flat = [&](int mode, int j, int k, int notail) {
        PointArgs pa{};
        pa.mode = mode;
        pa.j = j;
        pa.k = k;
        pa.m = mmax + 1;           // every column, m_max included, computes h_{j+1,j}
        pa.tol = btol;
        pa.notail = notail;
        pa.partials = E->d_partials;
        pa.counters = E->d_counters;
        C.point(pa);
    };
    auto matvec = [&](int j) {     // slot j+1 = dt H~ v_j (no fused dot)
        StageArgs a = stage_defaults();
        a.x = j - 1;
        a.y_out = j;
        a.src_slot = j;
        a.x_scale_slot = KRY_S + j;
        a.ch = dt;
        a.ck = 1.0;
        C.stage(a);
    };
    long long tot_sub = 0, tot_mv = 0;
    int max_dim = 0;
    std::vector<double> s(np), tau(np), e;
    std::vector<int> done(np), acc_j(np);
    for (int n = 0; n < nsteps; ++n) {
        launch_set_clock(E->d_probs, np, t + n * dt, dt, C.s);
        ++*C.launches;
        C.prologue(PRO_KRYLOV, mmax + 1);
        std::fill(s.begin(), s.end(), 0.0);
        std::fill(tau.begin(), tau.end(), 1.0);
        std::fill(done.begin(), done.end(), 0);
        for (int sub = 0;; ++sub) {
            // start vector: [U; eta e_p] on the first substep, [U; y] on later ones
            flat(0, 0, 0, sub == 0 ? 0 : 2);
            int rc = read_all();
            if (rc != EWV_OK) return rc;
            std::vector<int> grow(np, 0), accepted(np, 0);
            std::vector<double> acc_err(np, 0.0), anext(np, 0.0);
            int ngrow = 0;
            for (int p = 0; p < np; ++p) {
                if (done[p]) continue;
                tau[p] = std::min(tau[p], 1.0 - s[p]);
                if (kb[p][KRY_ACTIVE] == 0.0) {     // a zero start vector stays zero
                    s[p] = 1.0;
                    done[p] = 1;
                    continue;
                }
                grow[p] = 1;
                ++ngrow;
            }
            if (ngrow == 0) break;
            bool have_next = false;
            for (int j = 1; j <= mmax && ngrow > 0; ++j) {
                const int k0 = window > 0 ? std::max(1, j - window + 1) : 1;
                if (!have_next) {
                    matvec(j);
                    ++tot_mv;
                }
                flat(5, j, k0, 0);                 // <q_{j+1}, q_k0> -> tail_{j+1}, h_{k0,j}
                for (int k = k0; k <= j; ++k) flat(1, j, k, 0);
                have_next = false;
                if (j >= mmin && j < mmax + 1) {
                    matvec(j + 1);                 // A v_{j+1}: the estimate, reused by column j+1
                    flat(7, j + 1, 0, 0);          // |q_{j+2}|^2 -> KRY_AN
                    ++tot_mv;
                    have_next = true;
                }
                rc = read_all();
                if (rc != EWV_OK) return rc;
                for (int p = 0; p < np; ++p) {
                    if (!grow[p]) continue;
                    std::vector<double>& k = kb[p];
                    const double beta = k[KRY_BETA];
                    const double h = k[KRY_H + j * MAX_M + (j - 1)];
                    double ph1, ph2;
                    bool take = false;
                    if (!(h > btol)) {             // happy breakdown: the rest of the step at once
                        tau[p] = 1.0 - s[p];
                        phi_block(k.data(), j, tau[p], e, ph1, ph2);
                        acc_err[p] = 0.0;
                        take = true;
                    } else if (j >= mmin) {
                        // |A v_{j+1}|: grid part from the pass, tail J (s_{j+1} tail_{j+1}) here
                        const double sn = k[KRY_S + j + 1];
                        const double* tn = k.data() + KRY_T + j * MAX_P;
                        const int pp = E->probs[p].p;
                        double tt = 0.0;
                        for (int q = 0; q + 1 < pp; ++q) tt += (sn * tn[q + 1]) * (sn * tn[q + 1]);
                        anext[p] = std::sqrt(k[KRY_AN] + tt);
                        phi_block(k.data(), j, tau[p], e, ph1, ph2);
                        double er = beta * h * (std::fabs(ph1) + std::fabs(ph2) * anext[p]);
                        if (er <= tol * tau[p] * beta) {
                            acc_err[p] = er;
                            take = true;
                        } else if (j == mmax) {
                            for (int it = 0; it < 60 && !take; ++it) {
                                tau[p] *= std::max(0.2, 0.9 * std::pow(tol * tau[p] * beta / er, 1.0 / mmax));
                                phi_block(k.data(), j, tau[p], e, ph1, ph2);
                                er = beta * h * (std::fabs(ph1) + std::fabs(ph2) * anext[p]);
                                if (er <= tol * tau[p] * beta) {
                                    acc_err[p] = er;
                                    take = true;
                                }
                            }
                            if (!take)
                                return fail(err, EWV_ERR_NONFINITE, "adaptive Krylov: a substep did not meet the tolerance");
                        }
                    }
                    if (take) {
                        for (int r = 0; r < j; ++r) k[KRY_E + r] = e[r];
                        k[KRY_MEFF] = (double)j;
                        k[KRY_ACTIVE] = 0.0;
                        acc_j[p] = j;
                        accepted[p] = 1;
                        grow[p] = 0;
                        --ngrow;
                        rc = write(p);
                        if (rc != EWV_OK) return rc;
                    }
                }
            }
            // U <- beta V_j e on the grid (combine), the tail y <- beta sum_k e_k s_k tail_k here
            for (int p = 0; p < np; ++p)
                if (!accepted[p]) {
                    kb[p][KRY_SKIP] = 1.0;
                    int rc2 = write(p);
                    if (rc2 != EWV_OK) return rc2;
                }
            PointArgs pc{};
            pc.mode = 2;
            pc.m = mmax;
            C.point(pc);
            for (int p = 0; p < np; ++p) {
                std::vector<double>& k = kb[p];
                if (!accepted[p]) continue;
                const int j = acc_j[p], pp = E->probs[p].p;
                std::vector<double> y(MAX_P, 0.0);
                for (int kk = 1; kk <= j; ++kk)
                    for (int q = 0; q < pp; ++q)
                        y[q] += k[KRY_BETA] * k[KRY_E + kk - 1] * k[KRY_S + kk] * k[KRY_T + (kk - 1) * MAX_P + q];
                for (int q = 0; q < MAX_P; ++q) k[KRY_T + q] = y[q];
                s[p] += tau[p];
                const double er = acc_err[p];
                tau[p] *= er == 0.0 ? 2.0 : std::min(2.0, 0.9 * std::pow(tol * tau[p] * k[KRY_BETA] / er, 1.0 / j));
                max_dim = std::max(max_dim, j);
                ++tot_sub;
                if (s[p] >= 1.0) done[p] = 1;
                k[KRY_SKIP] = done[p] ? 1.0 : 0.0;
                int rc2 = write(p);
                if (rc2 != EWV_OK) return rc2;
            }
            for (int p = 0; p < np; ++p)
                if (!accepted[p] && !done[p]) {     // not reached here: every growing problem accepts
                    kb[p][KRY_SKIP] = 0.0;
                    int rc2 = write(p);
                    if (rc2 != EWV_OK) return rc2;
                }
            bool all = true;
            for (int p = 0; p < np; ++p) all = all && done[p];
            if (all) break;
        }
        C.record();
    }
    // leave no problem marked for the regular steps
    for (int p = 0; p < np; ++p) {
        kb[p][KRY_SKIP] = 0.0;
        int rc = write(p);
        if (rc != EWV_OK) return rc;
    }
    if (stats) {
        stats[0] = (int)tot_sub;
        stats[1] = (int)tot_mv;
        stats[2] = max_dim;
    }
    return check_launch(err);
}

int run_leapfrog(Ctx& C, std::vector<ewv_model*>& models, double t, double dt, int nsteps, int variant) {
    bool need_init = false;
    for (ewv_model* m : models) need_init = need_init || !m->lf_history_valid;
    const int wmask = C.E->dims == 3 ? 0x3D : 0xD;   // u, the w fields (and psi in 3D)
    const bool diff = variant == EWV_LEAPFROG_DIFFERENCE;
    if (diff && C.E->dims != 2) return fail(*C.err, EWV_ERR_UNSUPPORTED, "difference form: 2D only");
    if (need_init) {
        C.copy(0, 1, wmask, false);   // u and w of level n -> history (level n-1)
        if (diff) {                   // d^0 = u^0 - u^{-1} = 0 in the history's v field
            PointArgs pz{};
            pz.mode = 6;
            pz.dst = 1;
            pz.fmask = 0x2;
            C.point(pz);
        }
        for (ewv_model* m : models) m->lf_history_valid = true;
    }
    launch_set_clock(C.E->d_probs, C.E->nprob, t, dt, C.s);
    ++*C.launches;
    // step n reads level n from vector (n even ? 0 : 1) and writes level n+1 over the other
    int rc = C.step_loop(nsteps, EWV_METHOD_LEAPFROG, variant, dt, 0, 0, 0, 2, [&](int n) {
        const int cur = (n & 1) ? 1 : 0, prev = 1 - cur;
        C.prologue(PRO_LEAPFROG, 1);
        C.timed([&] {
        if (C.E->dims == 3 && C.E->precision == EWV_F32 && C.E->tma_variant != 1) {
            if (launch_leapfrog_tma3d(C.E->R, tma3d_warps(C.E), C.E->d_probs, C.E->d_tbase, C.E->nprob,
                                      C.E->ntiles_by[0], cur, prev, variant, dt, C.E->d_err, C.s) != 0)
                C.launch_failed = 1;
        } else if (C.E->dims == 3) {
            launch_leapfrog3d(C.E->precision, C.E->R, C.E->ntiles, C.E->d_probs, C.E->d_tile_prob,
                              cur, prev, variant, dt, C.s);
        } else if (C.E->precision == EWV_F32) {
            const int set = tma_map_set(30);
            if (launch_leapfrog_tma(C.E->R, C.E->d_probs, C.E->d_tbase + (size_t)set * (C.E->nprob + 1),
                                    C.E->nprob, C.E->ntiles_by[set], cur, prev, variant, dt, C.E->d_err,
                                    C.s) != 0)
                C.launch_failed = 1;
        } else {
            launch_leapfrog(C.E->precision, C.E->R, C.E->ntiles, C.E->d_probs, C.E->d_tile_prob,
                            cur, prev, variant, dt, C.s);
        }
        });
        C.record(prev);
    });
    if (rc != EWV_OK) return rc;
    // level n back into the state, n-1 into history (and d^n with it in the difference form)
    if (nsteps & 1) C.copy(1, 0, wmask | (diff ? 0x2 : 0), true);
    return check_launch(*C.err);
}

int precheck_engine_models(std::vector<ewv_model*>& models, int method, int mm, std::string& err) {
    for (ewv_model* m : models) {
        int rc = check_bound(m, method, mm, err);
        if (rc != EWV_OK) return rc;
        if (m->d.precision != models[0]->d.precision || m->d.fd_order != models[0]->d.fd_order)
            return fail(err, EWV_ERR_INVALID_ARG, "batched models must share precision and fd order");
    }
    return EWV_OK;
}

int dispatch_method(Ctx& C, std::vector<ewv_model*>& models, int method, double t, double dt,
                    int mm, int nsteps, int* info);

Engine* ensure_model_engine(ewv_model* m) {
    if (!m->engine) {
        m->engine = new Engine();
        m->engine->models.push_back(m);
        m->engine->precision = m->d.precision;
        m->engine->R = m->R;
    }
    return m->engine;
}

int take_pending_error(Engine* E, cudaStream_t s, std::string& err);

int dispatch(std::vector<ewv_model*>& models, Engine* E, cudaStream_t s, long long* launches,
             std::string& err, int method, double t, double dt, int mm, int nsteps, int* info) {
    if (nsteps < 0) return fail(err, EWV_ERR_INVALID_ARG, "nsteps < 0");
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t))
        return fail(err, EWV_ERR_INVALID_ARG, "dt must be positive and finite");
    int rc = precheck_engine_models(models, method, mm, err);
    if (rc != EWV_OK) return rc;
    rc = engine_ready(E, err);
    if (rc != EWV_OK) return rc;
    rc = take_pending_error(E, s, err);
    if (rc != EWV_OK) return rc;
    // With graphs on, run the call on the engine's own (capturable, non-blocking) stream,
    // ordered after the caller's stream and before whatever the caller enqueues next.
    cudaStream_t run_s = s;
    const bool own = E->graphs_enabled && !E->graphs_broken;
    if (own) {
        if (!E->cap) {
            CUDA_OR_FAIL(err, cudaStreamCreateWithFlags(&E->cap, cudaStreamNonBlocking));
            CUDA_OR_FAIL(err, cudaEventCreateWithFlags(&E->ev_in, cudaEventDisableTiming));
            CUDA_OR_FAIL(err, cudaEventCreateWithFlags(&E->ev_out, cudaEventDisableTiming));
        }
        CUDA_OR_FAIL(err, cudaEventRecord(E->ev_in, s));
        CUDA_OR_FAIL(err, cudaStreamWaitEvent(E->cap, E->ev_in, 0));
        run_s = E->cap;
    }
    Ctx C{E, run_s, launches, &err};
    rc = dispatch_method(C, models, method, t, dt, mm, nsteps, info);
    if (rc == EWV_OK && C.launch_failed)
        rc = fail(err, EWV_ERR_CUDA, "a stencil pass could not be launched (no usable TMA variant)");
    if (rc == EWV_OK) {
        // end of the call's work: scan the states for non-finite values and copy the error
        // word to the host without waiting; the next call (or ewv_sync) reports it
        launch_nonfinite_scan(E->precision, E->nchunks, E->d_probs, E->d_pbase, E->nprob, E->d_err, run_s);
        ++*launches;
        CUDA_OR_FAIL(err, cudaMemcpyAsync(E->h_err, E->d_err, sizeof(int), cudaMemcpyDeviceToHost, run_s));
        CUDA_OR_FAIL(err, cudaEventRecord(E->err_ev, run_s));
    }
    if (own) {
        cudaEventRecord(E->ev_out, run_s);
        cudaStreamWaitEvent(s, E->ev_out, 0);
    }
    return rc;
}

// Report an error word that an earlier call's GPU work left (see dispatch): 0 while none
// has reached the host.  On a nonzero word the call waits for the engine's work, then
// clears the word on both sides and returns TIMEOUT or NONFINITE.
int take_pending_error(Engine* E, cudaStream_t s, std::string& err) {
    if (!E || !E->h_err) return EWV_OK;
    if (*(volatile int*)E->h_err == 0) return EWV_OK;
    if (E->cap) CUDA_OR_FAIL(err, cudaStreamSynchronize(E->cap));
    CUDA_OR_FAIL(err, cudaStreamSynchronize(s));
    const int w = *(volatile int*)E->h_err;
    CUDA_OR_FAIL(err, cudaMemset(E->d_err, 0, sizeof(int)));
    *(volatile int*)E->h_err = 0;
    if (w & 1) return fail(err, EWV_ERR_TIMEOUT, "a bounded wait in a TMA pass or a Gram-Schmidt barrier timed out "
                                                 "during an earlier call");
    return fail(err, EWV_ERR_NONFINITE, "a non-finite value appeared in the state during an earlier call");
}

// Wait for every call enqueued on the engine, then report its error word.
int sync_engine(Engine* E, cudaStream_t s, std::string& err) {
    if (E && E->cap) CUDA_OR_FAIL(err, cudaStreamSynchronize(E->cap));
    CUDA_OR_FAIL(err, cudaStreamSynchronize(s));
    return take_pending_error(E, s, err);
}

int dispatch_method(Ctx& C, std::vector<ewv_model*>& models, int method, double t, double dt,
                    int mm, int nsteps, int* info) {
    switch (method) {
        case EWV_METHOD_FABER: {
            double g, c0, c1;
            ellipse_of(models[0], &g, &c0, &c1);
            if (models.size() > 1 && !models[0]->ellipse_override) {
                // one ellipse enclosing every model's spectrum: the widest
                double gb = 0, c0b = 0, c1b = 0, best = -1;
                for (ewv_model* m : models) {
                    double gg, a0, a1;
                    ellipse_of(m, &gg, &a0, &a1);
                    const double ai = gg * (1 - a1);
                    if (ai > best) {
                        best = ai;
                        gb = gg;
                        c0b = a0;
                        c1b = a1;
                    }
                }
                g = gb;
                c0 = c0b;
                c1 = c1b;
            }
            return run_faber(C, t, dt, mm, nsteps, g, c0, c1);
        }
        case EWV_METHOD_KRYLOV: return run_krylov(C, t, dt, mm, nsteps, info);
        case EWV_METHOD_KRYLOV_ADAPTIVE:
            return run_krylov_adaptive(C, t, dt, C.E->ad_tol, C.E->ad_mmin, C.E->ad_mmax, nsteps,
                                       C.E->ad_stats);
        case EWV_METHOD_HORK: return run_hork(C, t, dt, mm, nsteps);
        case EWV_METHOD_RK32:
        case EWV_METHOD_RK44: return run_rk(C, t, dt, method, nsteps);
        case EWV_METHOD_LEAPFROG: return run_leapfrog(C, models, t, dt, nsteps, models[0]->lf_variant);
        default: return fail(*C.err, EWV_ERR_INVALID_ARG, "unknown method %d", method);
    }
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

const char* ewv_version(void) { return kVersion; }

int ewv_create_model(const ewv_model_desc* desc, ewv_model_t* out) {
    if (!desc || !out) return EWV_ERR_INVALID_ARG;
    *out = nullptr;
    const ewv_model_desc& d = *desc;
    // extents up to 2^30 keep the pitch arithmetic below in int range; the 32-bit receiver
    // offsets bound the padded grid further
    if ((d.dims != 2 && d.dims != 3) || (d.dims == 3 && (d.nz < 2 || d.nz > (1 << 30))) ||
        d.nx < 2 || d.ny < 2 || d.nx > (1 << 30) || d.ny > (1 << 30) ||
        !(d.dx > 0) || (d.fd_order != 4 && d.fd_order != 8) ||
        d.pml_width < 0 || d.beta0 < 0 || (d.precision != EWV_F32 && d.precision != EWV_F64) ||
        d.nshots < 1 || d.src_taylor_p < 1 || d.src_taylor_p > MAX_P || d.max_receivers < 0)
        return EWV_ERR_INVALID_ARG;
    if (d.free_surface && d.fd_order != 8) return EWV_ERR_UNSUPPORTED;
    if (ensure_tables() != 0) return EWV_ERR_CUDA;
    ewv_model* m = new ewv_model();
    m->d = d;
    m->R = d.fd_order / 2;
    m->elem = d.precision == EWV_F64 ? 8 : 4;
    const int per128 = 128 / m->elem;
    m->pitch = ((d.nx + per128 - 1) / per128) * per128;
    m->nz = d.dims == 3 ? d.nz : 1;
    m->nfields = d.dims == 3 ? 6 : 4;
    m->field_elems = (size_t)m->nz * d.ny * m->pitch;
    m->vec_elems = (size_t)m->nfields * m->field_elems;
    if ((size_t)m->nz * d.ny * m->pitch > (size_t)INT32_MAX) {
        delete m;
        return EWV_ERR_INVALID_ARG;   // receiver offsets are 32-bit
    }
    m->shots.resize(d.nshots);
    const int nr = d.max_receivers > 0 ? d.max_receivers : 1;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->d_rec, sizeof(int) * (size_t)nr * d.nshots);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_nrec, sizeof(int) * (size_t)d.nshots);
    if (e == cudaSuccess) e = cudaMemset(m->d_nrec, 0, sizeof(int) * (size_t)d.nshots);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_sigma, sizeof(double) * (size_t)MAX_SIGMA * d.nshots);
    // beta at distance d = k/2 cells from the first ghost line (Sec. 2 profile), k = 0 .. 2 pml
    m->nbtab = 2 * d.pml_width + 1;
    {
        std::vector<float> bt((size_t)m->nbtab, 0.f);
        for (int k = 0; k < m->nbtab && d.pml_width > 0; ++k) {
            const double r = 1.0 - (0.5 * k) / d.pml_width;
            bt[k] = (float)(d.beta0 * r * r);
        }
        if (e == cudaSuccess) e = cudaMalloc(&m->d_btab, sizeof(float) * bt.size());
        if (e == cudaSuccess) e = cudaMemcpy(m->d_btab, bt.data(), sizeof(float) * bt.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&m->d_kry, sizeof(double) * (size_t)KRY_STRIDE * d.nshots);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_clk, sizeof(long long) * 4 * (size_t)d.nshots);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_tclk, sizeof(double) * 2 * (size_t)d.nshots);
    if (e == cudaSuccess) e = cudaMemset(m->d_sigma, 0, sizeof(double) * (size_t)MAX_SIGMA * d.nshots);
    if (e == cudaSuccess) e = cudaMemset(m->d_kry, 0, sizeof(double) * (size_t)KRY_STRIDE * d.nshots);
    if (e == cudaSuccess) e = cudaMemset(m->d_clk, 0, sizeof(long long) * 4 * (size_t)d.nshots);
    if (e == cudaSuccess) e = cudaMemset(m->d_tclk, 0, sizeof(double) * 2 * (size_t)d.nshots);
    if (e != cudaSuccess) {
        ewv_destroy_model(m);
        return EWV_ERR_CUDA;
    }
    *out = m;
    return EWV_OK;
}

int ewv_destroy_model(ewv_model_t m) {
    if (!m) return EWV_ERR_INVALID_ARG;
    delete m->engine;
    cudaFree(m->d_rec);
    cudaFree(m->d_nrec);
    cudaFree(m->d_sigma);
    cudaFree(m->d_btab);
    cudaFree(m->d_kry);
    cudaFree(m->d_clk);
    cudaFree(m->d_tclk);
    delete m;
    return EWV_OK;
}

int ewv_set_stream(ewv_model_t m, void* stream) {
    if (!m) return EWV_ERR_INVALID_ARG;
    m->stream = (cudaStream_t)stream;
    return EWV_OK;
}

int ewv_layout(ewv_model_t m, ewv_layout_info* out) {
    if (!m || !out) return EWV_ERR_INVALID_ARG;
    out->pitch = m->pitch;
    out->elem_bytes = m->elem;
    out->field_elems = m->field_elems;
    out->vector_bytes = m->vec_elems * m->elem;
    out->state_bytes = out->vector_bytes * m->d.nshots;
    out->params_bytes = m->field_elems * m->elem;
    out->compact_n = compact_n(m);
    return EWV_OK;
}

int ewv_workspace_bytes(ewv_model_t m, int method, int mm, size_t* bytes) {
    if (!m || !bytes) return EWV_ERR_INVALID_ARG;
    const int nv = vectors_needed(method, mm);
    if (nv < 0) return fail(m->err, EWV_ERR_INVALID_ARG, "unknown method %d", method);
    if (method == EWV_METHOD_KRYLOV && (mm < 1 || mm > MAX_M))
        return fail(m->err, EWV_ERR_INVALID_ARG, "Krylov m must be 1..%d", MAX_M);
    *bytes = (size_t)nv * m->vec_elems * m->elem * m->d.nshots;
    return EWV_OK;
}

int ewv_bind_buffers(ewv_model_t m, void* state, size_t state_bytes, void* params,
                     size_t params_bytes, void* work, size_t work_bytes) {
    if (!m) return EWV_ERR_INVALID_ARG;
    const size_t sb = m->vec_elems * m->elem * m->d.nshots;
    if (!state || state_bytes < sb || !aligned(state))
        return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "state needs %zu bytes, 256-B aligned", sb);
    if (!params || params_bytes < m->field_elems * m->elem || !aligned(params))
        return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "params needs %zu bytes, 256-B aligned",
                    m->field_elems * m->elem);
    if (work && !aligned(work))
        return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "work must be 256-B aligned");
    const bool params_changed = params != m->params;
    m->state = state;
    m->state_bytes = state_bytes;
    m->params = params;
    m->params_bytes = params_bytes;
    m->work = work_bytes ? work : nullptr;
    m->work_bytes = work ? work_bytes : 0;
    CUDA_OR_FAIL(m->err, cudaMemsetAsync(state, 0, sb, m->stream));
    if (m->work) CUDA_OR_FAIL(m->err, cudaMemsetAsync(m->work, 0, m->work_bytes, m->stream));
    if (params_changed) m->velocity_set = false;
    m->lf_history_valid = false;
    ++m->version;
    return EWV_OK;
}

int ewv_bind_workspace(ewv_model_t m, void* work, size_t work_bytes) {
    if (!m) return EWV_ERR_INVALID_ARG;
    if (work && !aligned(work))
        return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "work must be 256-B aligned");
    m->work = work_bytes ? work : nullptr;
    m->work_bytes = work ? work_bytes : 0;
    if (m->work) CUDA_OR_FAIL(m->err, cudaMemsetAsync(m->work, 0, m->work_bytes, m->stream));
    m->lf_history_valid = false;
    ++m->version;
    return EWV_OK;
}

int ewv_bind_seismogram(ewv_model_t m, void* seismo, size_t bytes, int capacity) {
    if (!m || capacity < 0) return EWV_ERR_INVALID_ARG;
    const size_t need = (size_t)capacity * m->d.max_receivers * m->elem * m->d.nshots;
    if (seismo && (bytes < need || !aligned(seismo)))
        return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "seismogram needs %zu bytes", need);
    m->seismo = seismo;
    m->seismo_bytes = bytes;
    m->capacity = seismo ? capacity : 0;
    ++m->version;
    return ewv_reset_recording(m);
}

int ewv_reset_recording(ewv_model_t m) {
    if (!m) return EWV_ERR_INVALID_ARG;
    for (int s = 0; s < m->d.nshots; ++s)
        CUDA_OR_FAIL(m->err, cudaMemsetAsync(m->d_clk + 4 * s + 1, 0, sizeof(long long), m->stream));
    return EWV_OK;
}

int ewv_reset_state(ewv_model_t m) {
    if (!m) return EWV_ERR_INVALID_ARG;
    if (!m->state) return fail(m->err, EWV_ERR_NOT_BOUND, "state not bound");
    CUDA_OR_FAIL(m->err, cudaMemsetAsync(m->state, 0, m->vec_elems * m->elem * m->d.nshots, m->stream));
    m->lf_history_valid = false;
    return ewv_reset_recording(m);
}

int ewv_set_velocity(ewv_model_t m, const double* c, size_t count) {
    if (!m || !c) return EWV_ERR_INVALID_ARG;
    const int nx = m->d.nx, ny = m->d.ny, nz = m->nz;
    if (count != (size_t)nx * ny * nz)
        return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "velocity count %zu != nx*ny*nz", count);
    if (!m->params) return fail(m->err, EWV_ERR_NOT_BOUND, "params buffer not bound");
    double cmax = 0.0;
    for (size_t i = 0; i < count; ++i) {
        if (!(c[i] > 0.0) || !std::isfinite(c[i]))
            return fail(m->err, EWV_ERR_INVALID_ARG, "velocity must be positive and finite");
        cmax = std::max(cmax, c[i]);
    }
    std::vector<char> buf(m->field_elems * m->elem, 0);
    for (size_t r = 0; r < (size_t)ny * nz; ++r)        // row r = k ny + j
        for (int i = 0; i < nx; ++i) {
            const double v = c[r * nx + i] * c[r * nx + i];
            if (m->elem == 8) ((double*)buf.data())[r * m->pitch + i] = v;
            else ((float*)buf.data())[r * m->pitch + i] = (float)v;
        }
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(m->params, buf.data(), buf.size(), cudaMemcpyHostToDevice, m->stream));
    CUDA_OR_FAIL(m->err, cudaStreamSynchronize(m->stream));
    m->c_max = cmax;
    m->velocity_set = true;
    return EWV_OK;
}

// Shared implementation: `pos` holds (x, y) or (x, y, z) per receiver; indices per axis are
// floor(pos / dx + 1/2) (nearest node), all bit-exact int32.
static int set_src_rec(ewv_model_t m, int shot, const double* spos, double f_peak, double t0,
                       double amp, int nrec, const double* rpos, int32_t* src_idx_out,
                       int32_t* rec_idx_out) {
    const int nd = m->d.dims;
    if (shot < 0 || shot >= m->d.nshots) return EWV_ERR_INVALID_ARG;
    if (nrec < 0 || nrec > m->d.max_receivers || (nrec > 0 && !rpos))
        return fail(m->err, EWV_ERR_INVALID_ARG, "nrec must be 0..max_receivers");
    if (!(f_peak > 0) || !std::isfinite(t0) || !std::isfinite(amp))
        return fail(m->err, EWV_ERR_INVALID_ARG, "bad wavelet parameters");
    const int ext[3] = {m->d.nx, m->d.ny, m->nz};
    auto node = [&](const double* pos, long long* idx) {
        for (int a = 0; a < nd; ++a) {
            const double f = std::floor(pos[a] / m->d.dx + 0.5);   // range-checked before the cast
            if (!(f >= 0.0 && f < (double)ext[a])) return false;
            idx[a] = (long long)f;
        }
        if (nd == 2) idx[2] = 0;
        return true;
    };
    long long si[3] = {0, 0, 0};
    if (!node(spos, si)) return fail(m->err, EWV_ERR_INVALID_ARG, "source outside the grid");
    std::vector<int> off(nrec);
    std::vector<int32_t> ij((size_t)nd * nrec);
    for (int r = 0; r < nrec; ++r) {
        long long ri[3] = {0, 0, 0};
        if (!node(rpos + (size_t)nd * r, ri))
            return fail(m->err, EWV_ERR_INVALID_ARG, "receiver %d outside the grid", r);
        off[r] = (int)((ri[2] * m->d.ny + ri[1]) * m->pitch + ri[0]);
        for (int a = 0; a < nd; ++a) ij[(size_t)nd * r + a] = (int32_t)ri[a];
    }
    Shot& s = m->shots[shot];
    s.has_src = true;
    s.si = (int)si[0];
    s.sj = (int)si[1];
    s.sk = (int)si[2];
    s.f_peak = f_peak;
    s.t0 = t0;
    s.amp = amp;
    s.rec_off = off;
    if (nrec > 0)
        CUDA_OR_FAIL(m->err, cudaMemcpy(m->d_rec + (size_t)shot * m->d.max_receivers, off.data(),
                                        sizeof(int) * nrec, cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(m->err, cudaMemcpy(m->d_nrec + shot, &nrec, sizeof(int), cudaMemcpyHostToDevice));
    if (src_idx_out)
        for (int a = 0; a < nd; ++a) src_idx_out[a] = (int32_t)si[a];
    if (rec_idx_out && nrec > 0) std::memcpy(rec_idx_out, ij.data(), sizeof(int32_t) * ij.size());
    ++m->version;
    return EWV_OK;
}

int ewv_set_source_receivers(ewv_model_t m, int shot, double sx, double sy, double f_peak,
                             double t0, double amp, int nrec, const double* rxy,
                             int32_t* src_idx_out, int32_t* rec_idx_out) {
    if (!m) return EWV_ERR_INVALID_ARG;
    if (m->d.dims != 2) return fail(m->err, EWV_ERR_INVALID_ARG, "3D model: use ewv_set_source_receivers3d");
    const double spos[2] = {sx, sy};
    return set_src_rec(m, shot, spos, f_peak, t0, amp, nrec, rxy, src_idx_out, rec_idx_out);
}

int ewv_set_source_receivers3d(ewv_model_t m, int shot, double sx, double sy, double sz,
                               double f_peak, double t0, double amp, int nrec, const double* rxyz,
                               int32_t* src_idx_out, int32_t* rec_idx_out) {
    if (!m) return EWV_ERR_INVALID_ARG;
    if (m->d.dims != 3) return fail(m->err, EWV_ERR_INVALID_ARG, "2D model: use ewv_set_source_receivers");
    const double spos[3] = {sx, sy, sz};
    return set_src_rec(m, shot, spos, f_peak, t0, amp, nrec, rxyz, src_idx_out, rec_idx_out);
}

int ewv_set_faber_ellipse(ewv_model_t m, double g, double c0, double c1) {
    if (!m || !(g > 0) || !std::isfinite(c0) || !std::isfinite(c1)) return EWV_ERR_INVALID_ARG;
    m->ellipse_override = true;
    m->eg = g;
    m->ec0 = c0;
    m->ec1 = c1;
    return EWV_OK;
}

int ewv_get_faber_ellipse(ewv_model_t m, double* g, double* c0, double* c1) {
    if (!m || !g || !c0 || !c1) return EWV_ERR_INVALID_ARG;
    if (!m->velocity_set && !m->ellipse_override) return fail(m->err, EWV_ERR_NOT_BOUND, "velocity not set");
    ellipse_of(m, g, c0, c1);
    return EWV_OK;
}

// ---- state transfer
// Compact host order: fields in turn, each [ez][ey][ex] row-major (its own extents).
static int pack_host(ewv_model* m, const double* h, std::vector<char>& buf) {
    const int ny = m->d.ny, P = m->pitch;
    buf.assign(m->vec_elems * m->elem, 0);
    size_t o = 0;
    for (int f = 0; f < m->nfields; ++f) {
        int ex, ey, ez;
        field_extent(m, f, &ex, &ey, &ez);
        for (int k = 0; k < ez; ++k)
            for (int j = 0; j < ey; ++j)
                for (int i = 0; i < ex; ++i) {
                    const size_t idx = (size_t)f * m->field_elems + ((size_t)k * ny + j) * P + i;
                    if (m->elem == 8) ((double*)buf.data())[idx] = h[o];
                    else ((float*)buf.data())[idx] = (float)h[o];
                    ++o;
                }
    }
    return EWV_OK;
}

static void unpack_host(ewv_model* m, const std::vector<char>& buf, double* h) {
    const int ny = m->d.ny, P = m->pitch;
    size_t o = 0;
    for (int f = 0; f < m->nfields; ++f) {
        int ex, ey, ez;
        field_extent(m, f, &ex, &ey, &ez);
        for (int k = 0; k < ez; ++k)
            for (int j = 0; j < ey; ++j)
                for (int i = 0; i < ex; ++i) {
                    const size_t idx = (size_t)f * m->field_elems + ((size_t)k * ny + j) * P + i;
                    h[o++] = m->elem == 8 ? ((const double*)buf.data())[idx]
                                          : (double)((const float*)buf.data())[idx];
                }
    }
}

int ewv_pack_vector(ewv_model_t m, const double* host, size_t n, void* dev) {
    if (!m || !host || !dev) return EWV_ERR_INVALID_ARG;
    if (n != compact_n(m)) return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "compact length %zu != %zu", n, compact_n(m));
    std::vector<char> buf;
    pack_host(m, host, buf);
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(dev, buf.data(), buf.size(), cudaMemcpyHostToDevice, m->stream));
    CUDA_OR_FAIL(m->err, cudaStreamSynchronize(m->stream));
    return EWV_OK;
}

int ewv_unpack_vector(ewv_model_t m, const void* dev, double* host, size_t n) {
    if (!m || !host || !dev) return EWV_ERR_INVALID_ARG;
    if (n != compact_n(m)) return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "compact length %zu != %zu", n, compact_n(m));
    std::vector<char> buf(m->vec_elems * m->elem);
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(buf.data(), dev, buf.size(), cudaMemcpyDeviceToHost, m->stream));
    CUDA_OR_FAIL(m->err, cudaStreamSynchronize(m->stream));
    unpack_host(m, buf, host);
    return EWV_OK;
}

int ewv_set_state(ewv_model_t m, int shot, const double* host, size_t n) {
    if (!m || shot < 0 || shot >= m->d.nshots) return EWV_ERR_INVALID_ARG;
    if (!m->state) return fail(m->err, EWV_ERR_NOT_BOUND, "state not bound");
    m->lf_history_valid = false;
    return ewv_pack_vector(m, host, n, (char*)m->state + (size_t)shot * m->vec_elems * m->elem);
}

int ewv_get_state(ewv_model_t m, int shot, double* host, size_t n) {
    if (!m || shot < 0 || shot >= m->d.nshots) return EWV_ERR_INVALID_ARG;
    if (!m->state) return fail(m->err, EWV_ERR_NOT_BOUND, "state not bound");
    return ewv_unpack_vector(m, (const char*)m->state + (size_t)shot * m->vec_elems * m->elem, host, n);
}

int ewv_apply_operator(ewv_model_t m, int transpose, const void* x, void* y) {
    if (!m || !x || !y || x == y) return EWV_ERR_INVALID_ARG;
    if (!aligned(x) || !aligned(y)) return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "x, y must be 256-B aligned");
    if (!m->params || !m->velocity_set) return fail(m->err, EWV_ERR_NOT_BOUND, "velocity not set");
    if (m->d.dims == 3 && transpose)
        return fail(m->err, EWV_ERR_UNSUPPORTED, "the 3D operator has no transpose pass");
    Engine* E = ensure_model_engine(m);
    ProblemDev P = make_problem(m, 0, 0);
    P.tmaps = nullptr;
    P.has_src = 0;
    P.state = const_cast<void*>(x);
    P.work = y;
    cudaFree(E->d_apply);
    E->d_apply = nullptr;
    CUDA_OR_FAIL(m->err, cudaMalloc(&E->d_apply, sizeof(ProblemDev) + sizeof(int) * P.ntiles));
    std::vector<int> tp(P.ntiles, 0);
    int* d_tp = (int*)((char*)E->d_apply + sizeof(ProblemDev));
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(E->d_apply, &P, sizeof(ProblemDev), cudaMemcpyHostToDevice, m->stream));
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(d_tp, tp.data(), sizeof(int) * P.ntiles, cudaMemcpyHostToDevice, m->stream));
    StageArgs a = stage_defaults();
    a.x = 0;
    a.y_out = 1;
    a.ch = 1.0;
    a.ck = 1.0;
    a.transpose = transpose ? 1 : 0;
    if (m->d.dims == 3) {
        launch_stage3d(m->d.precision, m->R, P.ntiles, E->d_apply, d_tp, a, m->stream);
    } else {
        launch_stage(m->d.precision, m->R, P.ntiles, E->d_apply, d_tp, a, m->stream);
    }
    ++m->launches;
    // keep the host copies alive until the copies complete
    CUDA_OR_FAIL(m->err, cudaStreamSynchronize(m->stream));
    return check_launch(m->err);
}

// ---- stepping (single model)
static int step_model(ewv_model_t m, int method, double t, double dt, int mm, int nsteps, int* info) {
    if (!m) return EWV_ERR_INVALID_ARG;
    std::vector<ewv_model*> models{m};
    Engine* E = ensure_model_engine(m);
    return dispatch(models, E, m->stream, &m->launches, m->err, method, t, dt, mm, nsteps, info);
}

int ewv_step_faber(ewv_model_t m, double t, double dt, int degree, int nsteps) {
    return step_model(m, EWV_METHOD_FABER, t, dt, degree, nsteps, nullptr);
}
int ewv_step_krylov(ewv_model_t m, double t, double dt, int mm, int nsteps, int* info) {
    return step_model(m, EWV_METHOD_KRYLOV, t, dt, mm, nsteps, info);
}
static int adaptive_call(std::vector<ewv_model*>& models, Engine* E, cudaStream_t s, long long* launches,
                         std::string& err, double t, double dt, double tol, int mmin, int mmax, int nsteps,
                         int* stats) {
    if (!(tol > 0.0) || mmin < 1 || mmax < mmin || mmax + 1 > MAX_M)
        return fail(err, EWV_ERR_INVALID_ARG, "adaptive Krylov: need tol > 0 and 1 <= m_min <= m_max <= %d",
                    MAX_M - 1);
    E->ad_tol = tol;
    E->ad_mmin = mmin;
    E->ad_mmax = mmax;
    E->ad_stats[0] = E->ad_stats[1] = E->ad_stats[2] = 0;
    const int rc = dispatch(models, E, s, launches, err, EWV_METHOD_KRYLOV_ADAPTIVE, t, dt, mmax, nsteps, nullptr);
    if (stats)
        for (int q = 0; q < 3; ++q) stats[q] = E->ad_stats[q];
    return rc;
}

int ewv_step_krylov_adaptive(ewv_model_t m, double t, double dt, double tol, int mmin, int mmax,
                             int nsteps, int* stats) {
    if (!m) return EWV_ERR_INVALID_ARG;
    std::vector<ewv_model*> models{m};
    Engine* E = ensure_model_engine(m);
    return adaptive_call(models, E, m->stream, &m->launches, m->err, t, dt, tol, mmin, mmax, nsteps, stats);
}

int ewv_step_rk(ewv_model_t m, double t, double dt, int scheme, int stages, int nsteps) {
    if (scheme != EWV_METHOD_HORK && scheme != EWV_METHOD_RK32 && scheme != EWV_METHOD_RK44)
        return m ? fail(m->err, EWV_ERR_INVALID_ARG, "scheme must be HORK, RK32 or RK44") : EWV_ERR_INVALID_ARG;
    return step_model(m, scheme, t, dt, stages, nsteps, nullptr);
}
int ewv_step_leapfrog(ewv_model_t m, double t, double dt, int nsteps) {
    return step_model(m, EWV_METHOD_LEAPFROG, t, dt, 1, nsteps, nullptr);
}
int ewv_set_leapfrog_variant(ewv_model_t m, int variant) {
    if (!m || (variant != EWV_LEAPFROG_AVERAGED && variant != EWV_LEAPFROG_LITERAL &&
               variant != EWV_LEAPFROG_DIFFERENCE))
        return EWV_ERR_INVALID_ARG;
    if (variant == EWV_LEAPFROG_DIFFERENCE && m->d.dims != 2)
        return fail(m->err, EWV_ERR_UNSUPPORTED, "the difference form of leap-frog is two-dimensional");
    // the difference form keeps d^n instead of u^{n-1}: a switch restarts the history
    if ((variant == EWV_LEAPFROG_DIFFERENCE) != (m->lf_variant == EWV_LEAPFROG_DIFFERENCE))
        m->lf_history_valid = false;
    m->lf_variant = variant;
    return EWV_OK;
}

int ewv_set_krylov_window(ewv_model_t m, int window) {
    if (!m || window < 0) return EWV_ERR_INVALID_ARG;
    if (m->kry_window != window) {
        m->kry_window = window;
        ++m->version;   // drops the captured step graphs
    }
    return EWV_OK;
}

int ewv_set_hork_form(ewv_model_t m, int form) {
    if (!m || (form != EWV_HORK_HORNER && form != EWV_HORK_LOW_STORAGE)) return EWV_ERR_INVALID_ARG;
    if (m->hork_form != form) {
        m->hork_form = form;
        ++m->version;   // drops the captured step graphs
    }
    return EWV_OK;
}

int ewv_set_storage_rounding(ewv_model_t m, int mode) {
    if (!m || (mode != EWV_STORE_FP32 && mode != EWV_STORE_BF16)) return EWV_ERR_INVALID_ARG;
    if (mode == EWV_STORE_BF16 && (m->d.precision != EWV_F32 || m->d.dims != 2))
        return fail(m->err, EWV_ERR_UNSUPPORTED, "bfloat16 storage rounding: 2D FP32 models only");
    m->store_bf16 = mode == EWV_STORE_BF16 ? 1 : 0;
    ++m->version;   // the engine picks the flag up on its next build
    return EWV_OK;
}

// ---- batches
int ewv_create_batch(const ewv_model_t* models, int n, ewv_batch_t* out) {
    if (!models || n < 1 || !out) return EWV_ERR_INVALID_ARG;
    ewv_batch* b = new ewv_batch();
    for (int i = 0; i < n; ++i) {
        if (!models[i]) {
            delete b;
            return EWV_ERR_INVALID_ARG;
        }
        b->models.push_back(models[i]);
    }
    for (int i = 1; i < n; ++i)
        if (models[i]->d.precision != models[0]->d.precision || models[i]->d.fd_order != models[0]->d.fd_order ||
            models[i]->d.free_surface != models[0]->d.free_surface) {
            delete b;
            return EWV_ERR_INVALID_ARG;
        }
    b->engine = new Engine();
    b->engine->models = b->models;
    b->engine->precision = models[0]->d.precision;
    b->engine->R = models[0]->R;
    *out = b;
    return EWV_OK;
}

int ewv_destroy_batch(ewv_batch_t b) {
    if (!b) return EWV_ERR_INVALID_ARG;
    delete b->engine;
    delete b;
    return EWV_OK;
}

int ewv_batch_set_stream(ewv_batch_t b, void* s) {
    if (!b) return EWV_ERR_INVALID_ARG;
    b->stream = (cudaStream_t)s;
    b->stream_set = true;
    return EWV_OK;
}

static int step_batch(ewv_batch_t b, int method, double t, double dt, int mm, int nsteps, int* info) {
    if (!b) return EWV_ERR_INVALID_ARG;
    cudaStream_t s = b->stream_set ? b->stream : b->models[0]->stream;
    long long dummy = 0;
    int rc = dispatch(b->models, b->engine, s, &dummy, b->err, method, t, dt, mm, nsteps, info);
    b->models[0]->launches += dummy;
    return rc;
}

int ewv_batch_step_faber(ewv_batch_t b, double t, double dt, int degree, int nsteps) {
    return step_batch(b, EWV_METHOD_FABER, t, dt, degree, nsteps, nullptr);
}
int ewv_batch_step_krylov(ewv_batch_t b, double t, double dt, int mm, int nsteps, int* info) {
    return step_batch(b, EWV_METHOD_KRYLOV, t, dt, mm, nsteps, info);
}
int ewv_batch_step_krylov_adaptive(ewv_batch_t b, double t, double dt, double tol, int mmin, int mmax,
                                   int nsteps, int* stats) {
    if (!b) return EWV_ERR_INVALID_ARG;
    cudaStream_t s = b->stream_set ? b->stream : b->models[0]->stream;
    long long dummy = 0;
    const int rc = adaptive_call(b->models, b->engine, s, &dummy, b->err, t, dt, tol, mmin, mmax, nsteps, stats);
    b->models[0]->launches += dummy;
    return rc;
}

int ewv_batch_step_rk(ewv_batch_t b, double t, double dt, int scheme, int stages, int nsteps) {
    if (scheme != EWV_METHOD_HORK && scheme != EWV_METHOD_RK32 && scheme != EWV_METHOD_RK44) return EWV_ERR_INVALID_ARG;
    return step_batch(b, scheme, t, dt, stages, nsteps, nullptr);
}
int ewv_batch_step_leapfrog(ewv_batch_t b, double t, double dt, int nsteps) {
    return step_batch(b, EWV_METHOD_LEAPFROG, t, dt, 1, nsteps, nullptr);
}

static int read_timing(Engine* E, cudaStream_t s, std::string& err, double* total_ms,
                       long long* count) {
    CUDA_OR_FAIL(err, cudaStreamSynchronize(s));
    for (auto& kv : E->graphs)
        if (harvest_graph_timing(E, kv.second, err) != EWV_OK) return EWV_ERR_CUDA;
    double tot = E->timing_acc_ms;
    for (size_t k = 0; k + 1 < E->events_used; k += 2) {
        float ms = 0.f;
        CUDA_OR_FAIL(err, cudaEventElapsedTime(&ms, E->events[k], E->events[k + 1]));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (count) *count = (long long)(E->events_used / 2) + E->timing_acc_n;
    E->events_used = 0;
    E->timing_acc_ms = 0.0;
    E->timing_acc_n = 0;
    return EWV_OK;
}

static int set_variant(Engine* E, int v) {
    if (v < -1 || v >= TMA_NUM_VARIANTS) return EWV_ERR_INVALID_ARG;
    if (E->tma_variant != v) {
        E->tma_variant = v;
        E->drop_graphs();   // captured steps hold the previous variant's launches
    }
    return EWV_OK;
}

static int get_variant(Engine* E, int* v, int* by, int* nw, int* nst, double* us) {
    if (!v) return EWV_ERR_INVALID_ARG;
    *v = E->tma_variant;
    int b = 0, w = 0, n = 0;
    if (E->tma_variant >= 0) tma_variant_describe(E->tma_variant, &b, &w, &n);
    if (by) *by = b;
    if (nw) *nw = w;
    if (nst) *nst = n;
    if (us)
        for (int k = 0; k < TMA_NUM_VARIANTS; ++k) us[k] = E->tma_variant_us[k];
    return EWV_OK;
}

int ewv_set_kernel_variant(ewv_model_t m, int v) {
    if (!m) return EWV_ERR_INVALID_ARG;
    return set_variant(ensure_model_engine(m), v);
}
int ewv_kernel_variant(ewv_model_t m, int* v, int* by, int* nw, int* nst, double* us) {
    if (!m) return EWV_ERR_INVALID_ARG;
    return get_variant(ensure_model_engine(m), v, by, nw, nst, us);
}
int ewv_batch_set_kernel_variant(ewv_batch_t b, int v) {
    if (!b) return EWV_ERR_INVALID_ARG;
    return set_variant(b->engine, v);
}
int ewv_batch_kernel_variant(ewv_batch_t b, int* v, int* by, int* nw, int* nst, double* us) {
    if (!b) return EWV_ERR_INVALID_ARG;
    return get_variant(b->engine, v, by, nw, nst, us);
}

int ewv_enable_graphs(ewv_model_t m, int enable) {
    if (!m) return EWV_ERR_INVALID_ARG;
    Engine* E = ensure_model_engine(m);
    E->graphs_enabled = enable != 0;
    return EWV_OK;
}

int ewv_batch_enable_graphs(ewv_batch_t b, int enable) {
    if (!b) return EWV_ERR_INVALID_ARG;
    b->engine->graphs_enabled = enable != 0;
    return EWV_OK;
}

int ewv_enable_kernel_timing(ewv_model_t m, int enable) {
    if (!m) return EWV_ERR_INVALID_ARG;
    Engine* E = ensure_model_engine(m);
    E->timing = enable != 0;
    E->events_used = 0;
    E->timing_acc_ms = 0.0;
    E->timing_acc_n = 0;
    return EWV_OK;
}

int ewv_kernel_timing(ewv_model_t m, double* total_ms, long long* launches) {
    if (!m || !m->engine) return EWV_ERR_INVALID_ARG;
    return read_timing(m->engine, m->stream, m->err, total_ms, launches);
}

int ewv_batch_enable_kernel_timing(ewv_batch_t b, int enable) {
    if (!b) return EWV_ERR_INVALID_ARG;
    b->engine->timing = enable != 0;
    b->engine->events_used = 0;
    b->engine->timing_acc_ms = 0.0;
    b->engine->timing_acc_n = 0;
    return EWV_OK;
}

int ewv_batch_kernel_timing(ewv_batch_t b, double* total_ms, long long* launches) {
    if (!b) return EWV_ERR_INVALID_ARG;
    return read_timing(b->engine, b->stream_set ? b->stream : b->models[0]->stream, b->err,
                       total_ms, launches);
}

// ---- discrete adjoint (FWI gradient) -------------------------------------------------
// Krylov step adjoint (the step-level linearisation of the Krylov row of the FWI gradient):
// cotangent exp(dt H)^T ybar by Arnoldi on dt H^T, and the m-gradient
//   dt sum_q w_q [exp((1 - tau_q) dt H)^T ybar]_v  G(x(tau_q dt)),  x(s) = [I 0] exp(s H~)[U; e_p],
// with 4-point Gauss-Legendre nodes tau_q and dense output of both Arnoldi bases.  Three
// descriptor views of the workspace (per shot, W_k = workspace vector k):
//   F (state W_0 = checkpoint, work W_1): forward basis q_1 = W_0, q_{k+1} = W_k; x(tau_q) -> W_{m+q}
//   A (state = cotangent, work W_{m+5}): adjoint basis q'_1 = cotangent, q'_{k+1} = W_{m+4+k};
//     y(1 - tau_q) -> W_{2m+4+q}; finally y(1) -> the cotangent
//   G (state = cotangent, work W_0): gradient passes, x(tau_q) = G vector m+q+1, y = 2m+5+q.
static int adjoint_krylov(ewv_model* m, Engine* E, double t, double dt, int mm, void* adj_state,
                          void* grad, const std::vector<ProblemDev>& base, const int* d_tp, int tb,
                          const void* xdense) {
    cudaStream_t s = m->stream;
    const int ns = m->d.nshots, prec = m->d.precision, R = m->R;
    const size_t vb = m->vec_elems * m->elem;
    const size_t per_shot = (m->work_bytes / ns) / vb;
    auto wvec = [&](int sh, int k) { return (char*)m->work + ((size_t)sh * per_shot + (size_t)k) * vb; };
    std::vector<ProblemDev> views(3 * (size_t)ns);
    for (int sh = 0; sh < ns; ++sh) {
        ProblemDev P = base[sh];
        P.pchunks = E->probs[sh].pchunks;
        P.pchunk_base = E->probs[sh].pchunk_base;
        ProblemDev F = P, A = P, G = P;
        F.state = wvec(sh, 0);
        F.work = wvec(sh, 1);
        A.state = (char*)adj_state + (size_t)sh * vb;
        A.work = wvec(sh, mm + 5);
        G.state = A.state;
        G.work = wvec(sh, 0);
        views[sh] = F;
        views[ns + sh] = A;
        views[2 * ns + sh] = G;
    }
    // FP32: the products of both Arnoldi processes take the persistent TMA passes (the forward
    // one the autotuned variant, the transposed one 64 x 18 tiles), each followed by a flat
    // pass forming <q_{j+1}, q_1> with the finalisation of the plain kernel's fused dot; the
    // tensor maps describe the F and A views and are rebuilt when the buffers change.  The
    // gradient passes take the TMA gradient pass when the caller built maps of the G view
    // (the cotangent and the workspace from vector 0).
    bool tma = prec == EWV_F32 && E->tma_variant >= 0 && E->d_tbase && E->nprob == ns &&
               per_shot >= (size_t)(2 * mm + 9);
    if (tma && (E->kexp_key_state != adj_state || E->kexp_key_work != m->work ||
                E->kexp_key_bytes != m->work_bytes || E->kexp_key_m != mm)) {
        std::vector<ProblemDev> fa(views.begin(), views.begin() + 2 * (size_t)ns);
        std::vector<int> wv(2 * (size_t)ns);
        for (int sh = 0; sh < ns; ++sh) {
            wv[sh] = (int)per_shot - 1;
            wv[ns + sh] = (int)per_shot - (mm + 5);
        }
        E->kexp_key_state = nullptr;
        if (build_tensor_maps(fa, R, wv, &E->d_kexp_maps) == 0) {
            E->kexp_key_state = adj_state;
            E->kexp_key_work = m->work;
            E->kexp_key_bytes = m->work_bytes;
            E->kexp_key_m = mm;
            E->kexp_tmaps.assign(2 * (size_t)ns, nullptr);
            for (int i = 0; i < 2 * ns; ++i) E->kexp_tmaps[i] = fa[i].tmaps;
        } else {
            tma = false;
        }
    }
    if (tma)
        for (int i = 0; i < 2 * ns; ++i) views[i].tmaps = E->kexp_tmaps[i];
    const bool tma_grad = prec == EWV_F32 && E->d_tbase && E->nprob == ns && base[0].tmaps != nullptr;
    const size_t bytes = sizeof(ProblemDev) * views.size();
    if (!E->d_kadj || E->d_kadj_bytes < bytes) {
        cudaFree(E->d_kadj);
        E->d_kadj = nullptr;
        CUDA_OR_FAIL(m->err, cudaMalloc(&E->d_kadj, bytes));
        E->d_kadj_bytes = bytes;
    }
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(E->d_kadj, views.data(), bytes, cudaMemcpyHostToDevice, s));
    const ProblemDev* vF = E->d_kadj;
    const ProblemDev* vA = E->d_kadj + ns;
    const ProblemDev* vG = E->d_kadj + 2 * ns;
    const double tol = prec == EWV_F64 ? 1e-14 : 1e-6;
    static const double kTau[4] = {0.069431844202973712, 0.33000947820757187,
                                   0.66999052179242813, 0.93056815579702629};
    static const double kW[4] = {0.17392742256872693, 0.32607257743127307,
                                 0.32607257743127307, 0.17392742256872693};
    const int fset = tma ? tma_map_set(tma_variant_tile_height_for(E->tma_variant, false)) : 0;
    const int trset = tma_map_set(18), gset = tma_map_set(30);
    const bool col = g_mgs_enabled && E->mgs_cpb > 0 && E->nprob == ns;
    auto arnoldi = [&](const ProblemDev* v, bool transpose) {
        PointArgs pn{};
        pn.mode = 0;
        pn.m = mm;
        pn.tol = tol;
        pn.notail = transpose ? 1 : 0;
        pn.partials = E->d_partials;
        pn.counters = E->d_counters;
        launch_point_flat(prec, E->nchunks, v, E->d_pbase, ns, pn, s);
        ++m->launches;
        for (int j = 1; j <= mm; ++j) {
            StageArgs a = stage_defaults();
            a.x = j - 1;
            a.y_out = j;
            a.d = 0;
            a.src_slot = transpose ? -1 : j;
            a.x_scale_slot = KRY_S + j;
            a.ch = dt;
            a.ck = 1.0;
            a.transpose = transpose ? 1 : 0;
            a.fin_mode = FIN_MATVEC;
            a.fin_j = j;
            a.m = mm;
            a.tol = tol;
            a.partials = E->d_partials;
            a.counters = E->d_counters;
            bool fused = true;
            if (col) {
                // the product without a dot (TMA pass in FP32), then the column kernel
                StageArgs b = a;
                b.d = -1;
                b.fin_mode = FIN_NONE;
                const int set = transpose ? trset : fset;
                const int* tbs = tma ? E->d_tbase + (size_t)set * (E->nprob + 1) : nullptr;
                int rc = 1;
                if (tma)
                    rc = transpose ? launch_transpose_tma(R, v, tbs, ns, E->ntiles_by[set], b, E->d_err, s)
                                   : launch_stage_tma(E->tma_variant, R, v, tbs, ns, E->ntiles_by[set], b, E->d_err, s);
                if (rc != 0) launch_stage(prec, R, tb, v, d_tp, b, s);
                ++m->launches;
                const int kmax = (j == mm) ? j - 1 : j;
                if (mgs_column(E, prec, v, ns, j, 1, kmax, mm, tol, s)) {
                    ++m->launches;
                    continue;
                }
                // the column kernel could not be launched: the flat dot, then the flat passes
                PointArgs pd{};
                pd.mode = 5;
                pd.j = j;
                pd.k = 1;
                pd.m = mm;
                pd.tol = tol;
                pd.partials = E->d_partials;
                pd.counters = E->d_counters;
                launch_point_flat(prec, E->nchunks, v, E->d_pbase, ns, pd, s);
                ++m->launches;
                fused = false;
            } else if (tma) {
                StageArgs b = a;
                b.d = -1;
                b.fin_mode = FIN_NONE;
                const int set = transpose ? trset : fset;
                const int* tbs = E->d_tbase + (size_t)set * (E->nprob + 1);
                const int rc = transpose
                                   ? launch_transpose_tma(R, v, tbs, ns, E->ntiles_by[set], b, E->d_err, s)
                                   : launch_stage_tma(E->tma_variant, R, v, tbs, ns, E->ntiles_by[set], b, E->d_err, s);
                if (rc == 0) {
                    PointArgs pd{};
                    pd.mode = 5;
                    pd.j = j;
                    pd.k = 1;
                    pd.m = mm;
                    pd.tol = tol;
                    pd.partials = E->d_partials;
                    pd.counters = E->d_counters;
                    launch_point_flat(prec, E->nchunks, v, E->d_pbase, ns, pd, s);
                    m->launches += 2;
                    fused = false;
                }
            }
            if (fused) {
                launch_stage(prec, R, tb, v, d_tp, a, s);
                ++m->launches;
            }
            const int kmax = (j == mm) ? j - 1 : j;
            for (int k = 1; k <= kmax; ++k) {
                PointArgs pm{};
                pm.mode = 1;
                pm.j = j;
                pm.k = k;
                pm.m = mm;
                pm.tol = tol;
                pm.partials = E->d_partials;
                pm.counters = E->d_counters;
                launch_point_flat(prec, E->nchunks, v, E->d_pbase, ns, pm, s);
                ++m->launches;
            }
        }
    };
    // dense output of a basis at ntau values of tau from one read of it: vectors dst .. dst + 3
    // (and, with final, the last tau into vector 0)
    auto dense = [&](const ProblemDev* v, const double* taus, int ntau, int dst, int final) {
        if (launch_expm_multi(v, ns, mm, s, taus, ntau, E->d_ecoef) != 0) return false;
        PointArgs pc{};
        pc.mode = 8;
        pc.m = mm;
        pc.nout = ntau - final;
        pc.final_out = final;
        pc.ecoef = E->d_ecoef;
        pc.dst = dst;
        launch_point_flat(prec, E->nchunks, v, E->d_pbase, ns, pc, s);
        m->launches += 2;
        return true;
    };
    if (xdense) {
        // the forward step's dense states, x(tau_q) [q][shot], into the slots where the
        // forward Arnoldi below would leave them
        for (int q = 0; q < 4; ++q)
            CUDA_OR_FAIL(m->err, cudaMemcpy2DAsync(wvec(0, mm + 1 + q), per_shot * vb,
                                                   static_cast<const char*>(xdense) + (size_t)q * ns * vb, vb, vb,
                                                   ns, cudaMemcpyDeviceToDevice, s));
    } else {
        // forward Arnoldi from the checkpoint (W_0 holds U^{n-1}), with the source of step n
        launch_set_clock(vF, ns, t, dt, s);
        launch_prologue(vF, ns, PRO_KRYLOV, mm, 0.0, 0.0, 0.0, s);
        m->launches += 2;
        arnoldi(vF, false);
        if (!dense(vF, kTau, 4, mm + 1, 0)) return fail(m->err, EWV_ERR_CUDA, "expm configuration failed");
    }
    // adjoint Arnoldi on dt H^T from the cotangent (no tail, no source)
    arnoldi(vA, true);
    // y(1 - tau_q) into vectors m+1 .. m+4 of A, and the new cotangent y(1) into the cotangent
    // buffer (the gradient passes below do not read it)
    const double taus_a[5] = {1.0 - kTau[0], 1.0 - kTau[1], 1.0 - kTau[2], 1.0 - kTau[3], 1.0};
    if (!dense(vA, taus_a, 5, mm + 1, 1)) return fail(m->err, EWV_ERR_CUDA, "expm configuration failed");
    // gradient: dt w_q y_v(1 - tau_q) G(x(tau_q))
    for (int q = 0; q < 4; ++q) {
        StageArgs gr = stage_defaults();
        gr.x = mm + 2 + q;
        gr.grad = grad;
        gr.gq = 2 * mm + 6 + q;
        gr.gscale = dt * kW[q];
        if (!tma_grad || launch_grad_tma(R, vG, E->d_tbase + (size_t)gset * (E->nprob + 1), ns, E->ntiles_by[gset],
                                         gr, E->d_err, s) != 0)
            launch_stage(prec, R, tb, vG, d_tp, gr, s);
        ++m->launches;
    }
    int rc = check_launch(m->err);
    if (rc != EWV_OK || !(tma || tma_grad)) return rc;
    // the TMA pipeline's timeout flag
    int herr = 0;
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(&herr, E->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(m->err, cudaStreamSynchronize(s));
    if (herr) {
        CUDA_OR_FAIL(m->err, cudaMemset(E->d_err, 0, sizeof(int)));
        return fail(m->err, EWV_ERR_TIMEOUT, "a bounded wait in a TMA pass or a Gram-Schmidt barrier timed out");
    }
    return EWV_OK;
}

// ---------------------------------------------------------------- exact Krylov adjoint
// Exact discrete adjoint of one Krylov step (reverse mode through the Arnoldi process; the
// passes are described in kernels_kadj.cu).  Views over the workspace wvec(i) of each shot:
// F (the forward Arnoldi: state = wvec(0) = the checkpoint copy, so q_k = wvec(k-1)) and A
// (state = the cotangent, work = wvec(0): vector i >= 1 is wvec(i-1), so q_k is vector k).
static int adjoint_krylov_exact(ewv_model* m, Engine* E, double t, double dt, int mm, void* adj_state,
                                void* grad, const std::vector<ProblemDev>& base, const int* d_tp, int tb) {
    cudaStream_t s = m->stream;
    const int ns = m->d.nshots, prec = m->d.precision, R = m->R, p = m->d.src_taylor_p;
    const size_t vb = m->vec_elems * m->elem;
    const size_t per_shot = (m->work_bytes / ns) / vb;
    if (per_shot < (size_t)(2 * mm + 4))
        return fail(m->err, EWV_ERR_WORKSPACE_TOO_SMALL, "exact Krylov adjoint needs 2m + 4 vectors");
    const int window = m->kry_window;
    auto wvec = [&](int sh, int k) { return (char*)m->work + ((size_t)sh * per_shot + (size_t)k) * vb; };
    if (!E->d_kbar || E->d_kbar_n < (size_t)ns * KB_STRIDE) {
        cudaFree(E->d_kbar);
        E->d_kbar = nullptr;
        CUDA_OR_FAIL(m->err, cudaMalloc(&E->d_kbar, sizeof(double) * (size_t)ns * KB_STRIDE));
        E->d_kbar_n = (size_t)ns * KB_STRIDE;
    }
    std::vector<ProblemDev> views(2 * (size_t)ns);
    for (int sh = 0; sh < ns; ++sh) {
        ProblemDev P = base[sh];
        P.pchunks = E->probs[sh].pchunks;
        P.pchunk_base = E->probs[sh].pchunk_base;
        P.kbar = E->d_kbar + (size_t)sh * KB_STRIDE;
        ProblemDev F = P, A = P;
        F.state = wvec(sh, 0);
        F.work = wvec(sh, 1);
        A.state = (char*)adj_state + (size_t)sh * vb;
        A.work = wvec(sh, 0);
        views[sh] = F;
        views[ns + sh] = A;
    }
    const size_t bytes = sizeof(ProblemDev) * views.size();
    if (!E->d_kadj || E->d_kadj_bytes < bytes) {
        cudaFree(E->d_kadj);
        E->d_kadj = nullptr;
        CUDA_OR_FAIL(m->err, cudaMalloc(&E->d_kadj, bytes));
        E->d_kadj_bytes = bytes;
    }
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(E->d_kadj, views.data(), bytes, cudaMemcpyHostToDevice, s));
    const ProblemDev* vF = E->d_kadj;
    const ProblemDev* vA = E->d_kadj + ns;
    const double tol = prec == EWV_F64 ? 1e-14 : 1e-6;
    // ---- forward Arnoldi of step n from the checkpoint (F view), exactly as run_krylov
    launch_set_clock(vF, ns, t, dt, s);
    launch_prologue(vF, ns, PRO_KRYLOV, mm, 0.0, 0.0, 0.0, s);
    m->launches += 2;
    {
        PointArgs pn{};
        pn.mode = 0;
        pn.m = mm;
        pn.tol = tol;
        pn.partials = E->d_partials;
        pn.counters = E->d_counters;
        launch_point_flat(prec, E->nchunks, vF, E->d_pbase, ns, pn, s);
        ++m->launches;
        for (int j = 1; j <= mm; ++j) {
            const int k0 = window > 0 ? std::max(1, j - window + 1) : 1;
            StageArgs a = stage_defaults();
            a.x = j - 1;
            a.y_out = j;
            a.d = k0 - 1;
            a.src_slot = j;
            a.x_scale_slot = KRY_S + j;
            a.ch = dt;
            a.ck = 1.0;
            a.fin_mode = FIN_MATVEC;
            a.fin_j = j;
            a.fin_k = k0;
            a.m = mm;
            a.tol = tol;
            a.partials = E->d_partials;
            a.counters = E->d_counters;
            launch_stage(prec, R, tb, vF, d_tp, a, s);
            ++m->launches;
            const int kmax = (j == mm) ? j - 1 : j;
            for (int k = k0; k <= kmax; ++k) {
                PointArgs pm{};
                pm.mode = 1;
                pm.j = j;
                pm.k = k;
                pm.m = mm;
                pm.tol = tol;
                pm.partials = E->d_partials;
                pm.counters = E->d_counters;
                launch_point_flat(prec, E->nchunks, vF, E->d_pbase, ns, pm, s);
                ++m->launches;
            }
        }
        if (launch_expm(vF, ns, mm, s) != 0) return fail(m->err, EWV_ERR_CUDA, "expm configuration failed");
        ++m->launches;
    }
    auto flat = [&](const KAdjArgs& ka) {
        launch_kadj_flat(prec, E->nchunks, vA, E->d_pbase, ns, ka, s);
        ++m->launches;
    };
    auto args = [&](int mode, int fin) {
        KAdjArgs ka{};
        ka.mode = mode;
        ka.fin = fin;
        ka.m = mm;
        ka.dot = -1;
        ka.partials = E->d_partials;
        ka.counters = E->d_counters;
        return ka;
    };
    // ---- <ybar, q_k> for the output's cotangents
    for (int k = 1; k <= mm; ++k) {
        KAdjArgs ka = args(KA_DOT, FK_STORE);
        ka.a = 0;
        ka.b = k;
        ka.slot = KB_D + k;
        flat(ka);
    }
    // ---- host: Hbar = L(H^T, ebar e_1^T), ebar_k = beta s_k <ybar, q_k>, beta_bar, Vbar = beta e ybar^T
    std::vector<double> kry((size_t)ns * KRY_STRIDE), kbh((size_t)ns * KB_STRIDE, 0.0);
    for (int sh = 0; sh < ns; ++sh)
        CUDA_OR_FAIL(m->err, cudaMemcpyAsync(kry.data() + (size_t)sh * KRY_STRIDE, base[sh].kry,
                                             sizeof(double) * KRY_STRIDE, cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(kbh.data(), E->d_kbar, sizeof(double) * (size_t)ns * KB_STRIDE,
                                         cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(m->err, cudaStreamSynchronize(s));
    int jmax = 0;
    for (int sh = 0; sh < ns; ++sh) {
        const double* k = kry.data() + (size_t)sh * KRY_STRIDE;
        double* kb = kbh.data() + (size_t)sh * KB_STRIDE;
        if (k[KRY_NONFINITE] != 0.0) return fail(m->err, EWV_ERR_NONFINITE, "non-finite value in the Arnoldi process");
        const int me = (int)k[KRY_MEFF];
        jmax = std::max(jmax, me);
        std::vector<double> dval(kb + KB_D, kb + KB_D + MAX_M + 2);
        std::fill(kb, kb + KB_STRIDE, 0.0);
        if (me <= 0) continue;
        const double beta = k[KRY_BETA];
        double bbar = 0.0;
        std::vector<double> ebar(me);
        for (int q = 1; q <= me; ++q) {
            const double sq = k[KRY_S + q], d = dval[q];
            ebar[q - 1] = beta * sq * d;
            bbar += k[KRY_E + q - 1] * sq * d;
            kb[KB_C + q] = beta * k[KRY_E + q - 1];
        }
        // L(X, Ebar) = upper-right block of expm([[X, Ebar], [0, X]]), X = H_me^T, Ebar = ebar e_1^T
        const int n2 = 2 * me;
        std::vector<double> big((size_t)n2 * n2, 0.0);
        for (int r = 0; r < me; ++r)
            for (int c = 0; c < me; ++c) {
                const double x = k[KRY_H + c * MAX_M + r];          // (H^T)_{rc} = H_{cr}
                big[(size_t)r * n2 + c] = x;
                big[(size_t)(me + r) * n2 + me + c] = x;
            }
        for (int r = 0; r < me; ++r) big[(size_t)r * n2 + me] = ebar[r];
        const std::vector<double> ex = host_expm(big, n2);
        for (int r = 0; r < me; ++r)
            for (int c = 0; c < me; ++c) kb[KB_HB + r * MAX_M + c] = ex[(size_t)r * n2 + me + c];
        kb[KB_BBAR] = bbar;
    }
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(E->d_kbar, kbh.data(), sizeof(double) * (size_t)ns * KB_STRIDE,
                                         cudaMemcpyHostToDevice, s));
    // ---- Vbar_k = beta e_k ybar
    for (int k = 1; k <= jmax; ++k) {
        KAdjArgs ka = args(KA_SCALE, FK_NONE);
        ka.a = 0;
        ka.b = mm + 1 + k;
        ka.slot = KB_C + k;
        flat(ka);
    }
    // ---- reverse sweep over the columns
    for (int j = jmax; j >= 1; --j) {
        const int k0 = window > 0 ? std::max(1, j - window + 1) : 1;
        KAdjArgs cp = args(KA_DOT, FK_COLPREP);      // <Vbar_{j+1}, q_{j+1}> -> hbar, wbar tail
        cp.j = j;
        cp.a = mm + 2 + j;
        cp.b = j + 1;
        flat(cp);
        KAdjArgs cs = args(KA_COLSET, FK_GSPREP);    // wbar, w; <wbar, q_j> -> step k = j
        cs.j = j;
        cs.dot = j;
        cs.fk = j;
        flat(cs);
        for (int k = j; k >= k0; --k) {
            KAdjArgs gs = args(KA_GS, k > k0 ? FK_GSPREP : FK_NONE);
            gs.j = j;
            gs.k = k;
            gs.k0 = k0;
            if (k > k0) {
                gs.dot = k - 1;
                gs.fk = k - 1;
            }
            flat(gs);
        }
        // w = A v_j: tail and source terms, Vbar_j += dt H^T wbar, grad += dt s_j wbar_v G(q_j)
        launch_kadj_src(vA, ns, prec, j, mm, dt, s);
        ++m->launches;
        StageArgs tr = stage_defaults();
        tr.transpose = 1;
        tr.x = 2 * mm + 3;
        tr.ch = dt;
        tr.a = mm + 1 + j;
        tr.ca = 1.0;
        tr.cak = 1.0;
        tr.acc_out = mm + 1 + j;
        launch_stage(prec, R, tb, vA, d_tp, tr, s);
        StageArgs gr = stage_defaults();
        gr.x = j;
        gr.grad = grad;
        gr.gq = 2 * mm + 3;
        gr.gscale = dt;
        gr.x_scale_slot = KRY_S + j;
        launch_stage(prec, R, tb, vA, d_tp, gr, s);
        m->launches += 2;
    }
    // ---- start: v_1 = x / beta, beta = |x|, x = [U; eta e_p], eta = |U|
    KAdjArgs st = args(KA_DOT, FK_START);
    st.a = mm + 2;
    st.b = 1;
    flat(st);
    flat(args(KA_OUT, FK_NONE));
    return check_launch(m->err);
}

int ewv_set_krylov_adjoint(ewv_model_t m, int mode) {
    if (!m) return EWV_ERR_INVALID_ARG;
    if (mode != EWV_KRYLOV_ADJOINT_EXACT && mode != EWV_KRYLOV_ADJOINT_EXPONENTIAL)
        return fail(m->err, EWV_ERR_INVALID_ARG, "unknown Krylov adjoint mode %d", mode);
    m->kry_adjoint = mode;
    return EWV_OK;
}

// One adjoint step; for the Krylov step, xdense (when set) holds the forward step's dense
// states and replaces the checkpoint (the adjoint of the step's exponential without the
// forward Arnoldi).
static int adjoint_step_impl(ewv_model_t m, int method, double t, double dt, int deg, const void* checkpoint,
                             const void* xdense, void* adj_state, void* grad) {
    if (!m || !(checkpoint || xdense) || !adj_state || !grad) return EWV_ERR_INVALID_ARG;
    if (xdense && method != EWV_METHOD_KRYLOV)
        return fail(m->err, EWV_ERR_INVALID_ARG, "dense states belong to the Krylov step");
    if (xdense) checkpoint = xdense;   // validated below like a checkpoint, never read as one
    if (m->d.dims == 3) return fail(m->err, EWV_ERR_UNSUPPORTED, "the adjoint is two-dimensional");
    if (method != EWV_METHOD_FABER && method != EWV_METHOD_HORK && method != EWV_METHOD_KRYLOV &&
        method != EWV_METHOD_LEAPFROG)
        return fail(m->err, EWV_ERR_UNSUPPORTED,
                    "adjoint implemented for the Faber, HORK, Krylov and leap-frog steps");
    const bool lf = method == EWV_METHOD_LEAPFROG;
    if (lf && m->lf_variant == EWV_LEAPFROG_LITERAL)
        return fail(m->err, EWV_ERR_UNSUPPORTED, "leap-frog adjoint: averaged damping of w only");
    if ((!lf && (deg < 1 || deg > (method == EWV_METHOD_KRYLOV ? MAX_M : MAX_DEG))) || !(dt > 0.0))
        return fail(m->err, EWV_ERR_INVALID_ARG, "degree / dimension out of range or dt <= 0");
    if (!aligned(checkpoint) || !aligned(adj_state) || !aligned(grad))
        return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "adjoint buffers must be 256-B aligned");
    int rc = check_bound(m, method == EWV_METHOD_KRYLOV ? EWV_METHOD_ADJOINT_KRYLOV
                            : lf                        ? EWV_METHOD_ADJOINT_LEAPFROG
                                                        : EWV_METHOD_ADJOINT_FABER,
                         deg, m->err);
    if (rc != EWV_OK) return rc;
    Engine* E = ensure_model_engine(m);
    rc = engine_ready(E, m->err);
    if (rc != EWV_OK) return rc;
    cudaStream_t s = m->stream;
    const int ns = m->d.nshots;
    const size_t vb = m->vec_elems * m->elem;
    const size_t per_shot = (m->work_bytes / ns) / vb;        // workspace vectors per shot
    // descriptors: vector 0 = the cotangent (adj_state), work = this model's workspace
    std::vector<ProblemDev> probs;
    int tb = 0;
    for (int sh = 0; sh < ns; ++sh) {
        ProblemDev P = make_problem(m, sh, tb);
        P.state = (char*)adj_state + (size_t)sh * vb;
        P.work = (char*)m->work + (size_t)sh * per_shot * vb;
        P.tmaps = nullptr;
        tb += P.ntiles;
        probs.push_back(P);
    }
    std::vector<int> tp(tb);
    for (int p = 0; p < ns; ++p)
        for (int k = 0; k < probs[p].ntiles; ++k) tp[probs[p].tile_base + k] = p;
    const size_t adj_bytes = sizeof(ProblemDev) * ns + sizeof(int) * (size_t)tb;
    if (adj_bytes > E->d_adj_bytes) {
        cudaFree(E->d_adj);
        E->d_adj = nullptr;
        E->d_adj_bytes = 0;
        CUDA_OR_FAIL(m->err, cudaMalloc(&E->d_adj, adj_bytes));
        E->d_adj_bytes = adj_bytes;
    }
    int* d_tp = (int*)((char*)E->d_adj + sizeof(ProblemDev) * ns);
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(E->d_adj, probs.data(), sizeof(ProblemDev) * ns,
                                         cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(m->err, cudaMemcpyAsync(d_tp, tp.data(), sizeof(int) * (size_t)tb,
                                         cudaMemcpyHostToDevice, s));
    // checkpoint U^{n-1} -> tape slot T_0 (workspace vector 1) of every shot
    if (!xdense)
        CUDA_OR_FAIL(m->err, cudaMemcpy2DAsync(m->work, per_shot * vb, checkpoint, vb, vb, ns,
                                               cudaMemcpyDeviceToDevice, s));
    const int R = m->R, prec = m->d.precision;
    // FP32: the forward-recompute passes (no transpose, no gradient) take the persistent TMA
    // pass, with tensor maps of the adjoint's buffers (rebuilt when the buffers change)
    bool tma_adj = prec == EWV_F32 && E->tma_variant >= 0 && E->d_tbase && E->nprob == ns;
    if (tma_adj) {
        if (E->adj_key_state != adj_state || E->adj_key_work != m->work || E->adj_key_bytes != m->work_bytes) {
            std::vector<int> wv((size_t)ns, (int)per_shot);
            E->adj_key_state = nullptr;
            if (build_tensor_maps(probs, R, wv, &E->d_adj_maps) == 0) {
                E->adj_key_state = adj_state;
                E->adj_key_work = m->work;
                E->adj_key_bytes = m->work_bytes;
                E->adj_tmaps.assign((size_t)ns, nullptr);
                for (int p = 0; p < ns; ++p) E->adj_tmaps[p] = probs[p].tmaps;
            } else {
                tma_adj = false;
                for (ProblemDev& P : probs) P.tmaps = nullptr;
            }
        } else {
            for (int p = 0; p < ns; ++p) probs[p].tmaps = E->adj_tmaps[p];
        }
        CUDA_OR_FAIL(m->err, cudaMemcpyAsync(E->d_adj, probs.data(), sizeof(ProblemDev) * ns,
                                             cudaMemcpyHostToDevice, s));
    }
    auto tset_of = [&](const StageArgs& sa) {
        return tma_map_set(tma_variant_tile_height_for(E->tma_variant, sa.a >= 0));
    };
    const int gset = tma_map_set(30), trset = tma_map_set(18);
    auto stage = [&](const StageArgs& sa) {
        if (tma_adj && !sa.transpose && sa.grad && sa.fin_mode == FIN_NONE && sa.d < 0 &&
            launch_grad_tma(R, E->d_adj, E->d_tbase + (size_t)gset * (E->nprob + 1), ns, E->ntiles_by[gset], sa,
                            E->d_err, s) == 0) {
            ++m->launches;
            return;
        }
        if (tma_adj && sa.transpose && !sa.grad && sa.fin_mode == FIN_NONE && sa.d < 0 &&
            launch_transpose_tma(R, E->d_adj, E->d_tbase + (size_t)trset * (E->nprob + 1), ns, E->ntiles_by[trset],
                                 sa, E->d_err, s) == 0) {
            ++m->launches;
            return;
        }
        if (tma_adj && !sa.transpose && !sa.grad && sa.fin_mode == FIN_NONE && sa.d < 0 &&
            launch_stage_tma(E->tma_variant, R, E->d_adj, E->d_tbase + (size_t)tset_of(sa) * (E->nprob + 1), ns,
                             E->ntiles_by[tset_of(sa)], sa, E->d_err, s) == 0) {
            ++m->launches;
            return;
        }
        launch_stage(prec, R, tb, E->d_adj, d_tp, sa, s);
        ++m->launches;
    };
    // launch errors, and the TMA pipeline's timeout flag when it ran
    auto adj_finish = [&]() {
        int rc2 = check_launch(m->err);
        if (rc2 != EWV_OK || !tma_adj) return rc2;
        int herr = 0;
        CUDA_OR_FAIL(m->err, cudaMemcpyAsync(&herr, E->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_OR_FAIL(m->err, cudaStreamSynchronize(s));
        if (herr) {
            CUDA_OR_FAIL(m->err, cudaMemset(E->d_err, 0, sizeof(int)));
            return fail(m->err, EWV_ERR_TIMEOUT, "a bounded wait in a TMA pass or a Gram-Schmidt barrier timed out");
        }
        return EWV_OK;
    };
    if (method == EWV_METHOD_KRYLOV)
        return xdense || m->kry_adjoint == EWV_KRYLOV_ADJOINT_EXPONENTIAL
                   ? adjoint_krylov(m, E, t, dt, deg, adj_state, grad, probs, d_tp, tb, xdense)
                   : adjoint_krylov_exact(m, E, t, dt, deg, adj_state, grad, probs, d_tp, tb);
    if (lf) {
        // tape (vector 1) = level n; q in vector 2, H^T q in vector 3; the cotangents of
        // w^{n-1} live in the second nshots vectors of adj_state
        void* a1 = (char*)adj_state + (size_t)ns * vb;
        launch_leapfrog_adjoint(prec, tb, E->d_adj, d_tp, 0, 2, 3, a1, dt, s);
        ++m->launches;
        StageArgs gr = stage_defaults();       // grad += (s lam_u) G(u^n, w^n)
        gr.x = 1;
        gr.grad = grad;
        gr.gq = 2;
        gr.gscale = 1.0;
        stage(gr);
        StageArgs tr = stage_defaults();       // H^T q
        tr.transpose = 1;
        tr.x = 2;
        tr.ch = 1.0;
        tr.ck = 1.0;
        tr.y_out = 3;
        stage(tr);
        launch_leapfrog_adjoint(prec, tb, E->d_adj, d_tp, 1, 2, 3, a1, dt, s);
        ++m->launches;
        return adj_finish();
    }
    if (method == EWV_METHOD_HORK) {
        // u^{n+1} = sum_i w_i k_i, k_i = (I + dt H~) k_{i-1}; tape T_k = k_k = vector k+1
        const std::vector<double> lam = hork_lambdas(deg);
        auto w = [&](int i) { return i <= deg - 2 ? lam[i] : (i == deg - 1 ? 0.0 : lam[deg - 1]); };
        launch_set_clock(E->d_adj, ns, t, dt, s);
        launch_prologue(E->d_adj, ns, 3 /* HORK */, deg, 0.0, 0.0, 0.0, s);
        m->launches += 2;
        for (int j = 1; j <= deg - 1; ++j) {
            StageArgs sa = stage_defaults();
            sa.x = j;
            sa.y_out = j + 1;
            sa.src_slot = j - 1;
            sa.cx = 1.0;
            sa.ch = dt;
            sa.ck = 1.0;
            stage(sa);
        }
        // r_m = w_m ybar (not stored); r_{i-1} = w_{i-1} ybar + (I + dt H)^T r_i
        auto rbuf = [&](int k) { return k == 0 ? 0 : deg + 1 + ((deg - 1 - k) % 2); };
        for (int i = deg; i >= 1; --i) {
            const double sc = (i == deg) ? w(deg) : 1.0;
            StageArgs gr = stage_defaults();
            gr.x = i;                              // k_{i-1}
            gr.grad = grad;
            gr.gq = (i == deg) ? 0 : rbuf(i);
            gr.gscale = dt * sc;
            stage(gr);
            StageArgs tr = stage_defaults();
            tr.transpose = 1;
            tr.x = (i == deg) ? 0 : rbuf(i);
            tr.cx = sc;
            tr.ch = dt * sc;
            tr.a = 0;
            tr.ca = w(i - 1);
            tr.cak = 1.0;
            tr.acc_out = (i == 1 && deg == 1) ? deg + 1 : rbuf(i - 1);
            stage(tr);
        }
        if (deg == 1) {
            PointArgs pa{};
            pa.mode = 3;
            pa.src = deg + 1;
            pa.dst = 0;
            pa.fmask = 0xF;
            launch_point(prec, tb, E->d_adj, d_tp, pa, s);
            ++m->launches;
        }
        return adj_finish();
    }
    double g, c0, c1;
    ellipse_of(m, &g, &c0, &c1);
    auto key = std::make_tuple(dt, deg, g, c0, c1);
    auto it = E->faber_cache.find(key);
    if (it == E->faber_cache.end()) {
        launch_faber_coeffs(dt, g, c0, c1, deg, E->d_coef, s);
        ++m->launches;
        std::vector<double> a(deg + 1);
        CUDA_OR_FAIL(m->err, cudaMemcpyAsync(a.data(), E->d_coef, sizeof(double) * (deg + 1),
                                             cudaMemcpyDeviceToHost, s));
        CUDA_OR_FAIL(m->err, cudaStreamSynchronize(s));
        it = E->faber_cache.emplace(key, a).first;
    }
    const std::vector<double>& a = it->second;
    auto cprime = [&](int k) { return k <= 1 ? 0.0 : (k == 2 ? 2.0 * c1 : c1); };
    launch_set_clock(E->d_adj, ns, t, dt, s);
    launch_prologue(E->d_adj, ns, 1 /* Faber */, deg, g, c0, c1, s);
    m->launches += 2;
    // recompute the forward vectors p_1..p_{m-1} of this step into the tape (T_k = vector k+1)
    for (int j = 1; j <= deg - 1; ++j) {
        StageArgs sa = stage_defaults();
        sa.x = j;
        sa.u = j >= 2 ? j - 1 : -1;
        sa.y_out = j + 1;
        sa.src_slot = j - 1;
        sa.cx = -c0;
        sa.ch = 1.0 / g;
        sa.cu = -cprime(j);
        sa.ck = 1.0;
        stage(sa);
    }
    // reverse recurrence; ybar is vector 0, q_{m-k} lives in Q[(k-1) % 3] (vectors m+1..m+3)
    auto qbuf = [&](int jj) { return jj == 0 ? 0 : deg + 1 + ((deg - jj - 1) % 3); };
    for (int j = deg; j >= 1; --j) {
        // gradient: (1/gamma) q_{j,v} G(p_{j-1}); q_m = a_m ybar is not stored
        StageArgs gr = stage_defaults();
        gr.x = j;                              // T_{j-1}
        gr.grad = grad;
        gr.gq = (j == deg) ? 0 : qbuf(j);
        gr.gscale = (j == deg) ? a[deg] / g : 1.0 / g;
        stage(gr);
        // q_{j-1} = a_{j-1} ybar + B^T q_j - c'_{j+1} q_{j+1}
        StageArgs tr = stage_defaults();
        tr.transpose = 1;
        tr.a = 0;
        tr.cak = 1.0;
        if (j == deg) {
            tr.x = 0;
            tr.cx = -c0 * a[deg];
            tr.ch = a[deg] / g;
            tr.ca = a[deg - 1];
        } else if (j == deg - 1) {
            tr.x = qbuf(j);
            tr.cx = -c0;
            tr.ch = 1.0 / g;
            tr.ca = a[j - 1] - cprime(j + 1) * a[deg];
        } else {
            tr.x = qbuf(j);
            tr.u = qbuf(j + 1);
            tr.cau = -cprime(j + 1);
            tr.cx = -c0;
            tr.ch = 1.0 / g;
            tr.ca = a[j - 1];
        }
        // degree 1: q_0 cannot overwrite ybar while ybar is read with a halo
        tr.acc_out = (j == 1 && deg == 1) ? deg + 1 : qbuf(j - 1);
        stage(tr);
    }
    if (deg == 1) {
        PointArgs pa{};
        pa.mode = 3;
        pa.src = deg + 1;
        pa.dst = 0;
        pa.fmask = 0xF;
        launch_point(prec, tb, E->d_adj, d_tp, pa, s);
        ++m->launches;
    }
    return adj_finish();
}

int ewv_adjoint_step(ewv_model_t m, int method, double t, double dt, int deg,
                     const void* checkpoint, void* adj_state, void* grad) {
    return adjoint_step_impl(m, method, t, dt, deg, checkpoint, nullptr, adj_state, grad);
}

int ewv_adjoint_step_krylov_dense(ewv_model_t m, double t, double dt, int mdim, const void* dense,
                                  void* adj_state, void* grad) {
    if (!m || !dense) return EWV_ERR_INVALID_ARG;
    return adjoint_step_impl(m, EWV_METHOD_KRYLOV, t, dt, mdim, nullptr, dense, adj_state, grad);
}

int ewv_step_krylov_dense(ewv_model_t m, double t, double dt, int mdim, void* dense) {
    if (!m || !dense) return EWV_ERR_INVALID_ARG;
    if (!aligned(dense)) return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "dense buffer must be 256-B aligned");
    Engine* E = ensure_model_engine(m);
    E->kry_dense = dense;
    const int rc = step_model(m, EWV_METHOD_KRYLOV, t, dt, mdim, 1, nullptr);
    E->kry_dense = nullptr;
    return rc;
}

int ewv_adjoint_inject(ewv_model_t m, void* adj_state, const void* values) {
    if (!m || !adj_state || !values) return EWV_ERR_INVALID_ARG;
    const int ns = m->d.nshots, nr = m->d.max_receivers;
    // lambda_u[rec] += values[shot][rec]; receivers of one shot are added in order
    if (nr == 0) return EWV_OK;
    if (!aligned(adj_state)) return fail(m->err, EWV_ERR_BAD_SIZE_OR_ALIGNMENT, "adj_state must be 256-B aligned");
    launch_inject(m->d.precision, adj_state, (long long)m->vec_elems, values, m->d_rec, m->d_nrec, ns,
                  nr, m->stream);
    ++m->launches;
    return check_launch(m->err);
}

int ewv_sum_shot_fields(ewv_model_t m, const void* per_shot, void* out) {
    if (!m || !per_shot || !out) return EWV_ERR_INVALID_ARG;
    launch_sum_shots(m->d.precision, per_shot, out, (long long)m->field_elems, m->d.nshots, m->stream);
    ++m->launches;
    return check_launch(m->err);
}

int ewv_checkpoint_stride(int nsteps, int budget, int* stride) {
    if (nsteps < 0 || budget < 1 || !stride) return EWV_ERR_INVALID_ARG;
    *stride = nsteps <= budget ? 1 : (nsteps + budget - 1) / budget;
    return EWV_OK;
}

const char* ewv_last_error(ewv_model_t m) { return m ? m->err.c_str() : "null handle"; }
const char* ewv_batch_last_error(ewv_batch_t b) { return b ? b->err.c_str() : "null handle"; }

int ewv_launch_count(ewv_model_t m, long long* count) {
    if (!m || !count) return EWV_ERR_INVALID_ARG;
    *count = m->launches;
    return EWV_OK;
}

int ewv_sync(ewv_model_t m) {
    if (!m) return EWV_ERR_INVALID_ARG;
    return sync_engine(m->engine, m->stream, m->err);
}

int ewv_batch_sync(ewv_batch_t b) {
    if (!b) return EWV_ERR_INVALID_ARG;
    cudaStream_t s = b->stream_set ? b->stream : b->models[0]->stream;
    return sync_engine(b->engine, s, b->err);
}

int ewv_debug_set_wait_limit(unsigned long long ns) {
    if (ns > 1000000000ull) return EWV_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return EWV_ERR_CUDA;
    return set_tma_wait_limit_ns(ns) == 0 && set_mgs_wait_limit_ns(ns) == 0 ? EWV_OK : EWV_ERR_CUDA;
}

int ewv_debug_set_column_kernel(int enable) {
    if (cudaDeviceSynchronize() != cudaSuccess) return EWV_ERR_CUDA;
    g_mgs_enabled = enable != 0;
    return EWV_OK;
}

}  // extern "C"
