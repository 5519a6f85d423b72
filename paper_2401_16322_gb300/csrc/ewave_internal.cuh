// Internal declarations shared by the library's translation units (not part of the ABI).
//
// Data model.  A "problem" is one shot of one velocity model: its own state vector(s) on
// the padded grid plus a pointer to the model's c^2.  Every launch of a grid-sized kernel
// covers all problems of an engine (one model's shots, or a batch of models of uneven
// sizes) through a tile work list: block b handles tile (b - tile_base[p]) of problem
// p = tile_problem[b].  Per-problem scalars that kernels produce and consume (source
// scalars of each pass, Krylov/Hessenberg data, reduction partials, step clocks) live in
// small library-owned device arrays.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ewv {

// Tile of outputs per block (x contiguous) and block shape.
constexpr int BX = 64;
constexpr int BY = 16;
constexpr int TPX = 32;   // threads in x
constexpr int TPY = 8;    // threads in y
constexpr int NTHREADS = TPX * TPY;
constexpr int VX = BX / TPX;   // outputs per thread in x
constexpr int VY = BY / TPY;   // outputs per thread in y

constexpr int KC3 = 32;          // 3D: z planes per tile (a block marches down KC3 planes)
constexpr int PCHUNK = 8192;     // elements per block of the flat pointwise passes

constexpr int MAX_M = 48;        // Krylov dimension limit (EWV_MAX_KRYLOV_M)
constexpr int MAX_DEG = 128;     // Faber degree limit
constexpr int MAX_P = 24;        // augmented tail length limit
constexpr int MAX_SIGMA = 160;   // per-step source-scalar slots

// Per-problem Krylov scalar block (doubles), offsets.
constexpr int KRY_H = 0;                                  // (MAX_M+1) x MAX_M Hessenberg
constexpr int KRY_S = KRY_H + (MAX_M + 1) * MAX_M;        // slot scales s_k, k = 1..MAX_M+1
constexpr int KRY_T = KRY_S + (MAX_M + 2);                // tails Vt[k][MAX_P], k = 1..MAX_M+1
constexpr int KRY_W = KRY_T + (MAX_M + 2) * MAX_P;        // W scalars (source column values)
constexpr int KRY_E = KRY_W + MAX_P;                      // exp(H_m) e_1
constexpr int KRY_BETA = KRY_E + MAX_M;                   // |x|
constexpr int KRY_MEFF = KRY_BETA + 1;                    // effective dimension (as double)
constexpr int KRY_ACTIVE = KRY_MEFF + 1;                  // 1 while Arnoldi continues
constexpr int KRY_NONFINITE = KRY_ACTIVE + 1;             // 1 if a NaN/Inf was seen
constexpr int KRY_SKIP = KRY_NONFINITE + 1;               // adaptive step: 1 = not in this substep
constexpr int KRY_AN = KRY_SKIP + 1;                      // adaptive step: |q|^2 of a stored slot
constexpr int KRY_STRIDE = ((KRY_AN + 1 + 31) / 32) * 32;

struct ProblemDev {
    int nx, ny, pitch, fs;
    int pml, src_i, src_j, nrec;
    int tiles_x, tiles_y, tile_base, ntiles;
    int rec_stride, capacity, p, has_src;
    int shot, pad_;       // shot index inside its model (per-shot caller arrays)
    int nz, nfields;      // 2D: 1 and 4 (u, v, w_x, w_y); 3D: nz and 6 (w_z, psi added)
    int src_k, tiles_z;   // 3D: source plane, tiles along z (KC3 planes each); 2D: 0, 1
    int pchunks, pchunk_base;   // flat pointwise passes: chunks of this problem's vector, first
    int nbtab, pad2;      // entries of btab
    double beta0, inv_dx, inv_dx2, inv_pml;
    double f_peak, t0, amp;
    long long field_stride, vec_stride;
    void* state;          // vector 0 (this shot)
    void* work;           // vector 1 (vectors 1.. are consecutive)
    const void* c2;
    double* sigma;        // [MAX_SIGMA] source scalars of the current step's passes
    const int* rec_off;   // [nrec] (k*ny + j)*pitch + i
    void* seismo;         // [capacity][rec_stride] of this shot
    double* kry;          // [KRY_STRIDE]
    long long* clk;       // [4]: step within call, recording cursor, (unused), (unused)
    double* tclk;         // [2]: t_start, dt of the current call
    const void* tmaps;    // FP32: this problem's TMA tensor maps (kernels_tma.cu), else null
    const float* btab;    // beta0 (1 - d/delta)^2 at distances d = k/2 cells, k < nbtab (FP32)
    float fbeta0, finv_pml, finv_dx, finv_dx2;   // FP32 copies of the damping / grid constants
    double* kbar;         // exact Krylov adjoint: [KB_STRIDE] reverse-sweep scalars, else null
};

// Per-problem scalar block of the exact Krylov adjoint (doubles), offsets (kernels_kadj.cu).
constexpr int KB_HB = 0;                                  // Hbar, (MAX_M+1) x MAX_M, row k-1, col j-1
constexpr int KB_VT = KB_HB + (MAX_M + 1) * MAX_M;        // tails of Vbar_k, k = 1..MAX_M+1
constexpr int KB_WT = KB_VT + (MAX_M + 2) * MAX_P;        // tail of wbar
constexpr int KB_CT = KB_WT + MAX_P;                      // tail of the reconstructed w
constexpr int KB_D = KB_CT + MAX_P;                       // <ybar, q_k> (grid), k = 1..MAX_M+1
constexpr int KB_C = KB_D + MAX_M + 2;                    // beta e_k, k = 1..MAX_M+1
constexpr int KB_HBAR = KB_C + MAX_M + 2;                 // hbar of the current Gram-Schmidt step
constexpr int KB_HCOL = KB_HBAR + 1;                      // hbar of the column's normalisation
constexpr int KB_BBAR = KB_HCOL + 1;                      // beta bar
constexpr int KB_EBAR = KB_BBAR + 1;                      // eta bar
constexpr int KB_OA = KB_EBAR + 1;                        // output: lambda = a Vbar_1 + b q_1
constexpr int KB_OB = KB_OA + 1;
constexpr int KB_STRIDE = ((KB_OB + 1 + 31) / 32) * 32;

// Arguments of the exact Krylov adjoint's flat passes (kernels_kadj.cu).  Vector indices in
// the adjoint view: 0 = the cotangent (ybar in, lambda out), k = q_k (k = 1..m+1, the
// recomputed forward basis), m+1+k = Vbar_k, 2m+3 = wbar, 2m+4 = the reconstructed w.
enum { KA_DOT = 0, KA_SCALE = 1, KA_COLSET = 2, KA_GS = 3, KA_OUT = 4 };
enum { FK_NONE = 0, FK_STORE = 1, FK_COLPREP = 2, FK_GSPREP = 3, FK_START = 4 };
struct KAdjArgs {
    int mode, fin;
    int j, k, k0, m;      // column, Gram-Schmidt index, window start of the column, dimension
    int a, b;             // KA_DOT / KA_SCALE: vector indices (KA_SCALE: b = a * kb[slot])
    int slot;             // kb slot (FK_STORE target, KA_SCALE coefficient)
    int fk;               // Gram-Schmidt index the FK_GSPREP finalisation prepares
    int dot;              // KA_COLSET / KA_GS: vector index of the fused dot's partner (-1: none)
    double* partials;
    unsigned int* counters;
};
void launch_kadj_flat(int precision, int nchunks, const ProblemDev* probs, const int* pbase,
                      int nprob, const KAdjArgs& ka, cudaStream_t s);
// Source and tail terms of the reverse matrix-vector product of column j (one thread per problem).
void launch_kadj_src(const ProblemDev* probs, int nprob, int precision, int j, int m, double dt,
                     cudaStream_t s);

// Arguments of the fused stencil-stage kernel (see kernels_stencil.cu).
struct StageArgs {
    int x, u, a, y_out, acc_out;     // vector indices (-1 = none)
    int d;                           // dot partner vector (-1 = none)
    int src_slot;                    // sigma slot added at the source node (-1 = none)
    int x_scale_slot;                // -1 or KRY_S index + k: X multiplied by kry[slot]
    int fin_mode, fin_j, fin_k;      // last-block finalisation (Krylov), see kernels_aux
    int transpose;                   // 0: H, 1: H^T
    double cx, ch, cu, ck, ca, cau, cak, cay, cax;
    double* partials;                // per-block partial dot products (global index)
    unsigned int* counters;          // per-problem arrival counters
    double tol;                      // breakdown tolerance (Krylov)
    int m;                           // Krylov dimension of this step
    double dt;
    void* grad;                      // gradient mode: grad += gscale q_v G(X), per-shot fields
    int gq;                          // vector index of q (its v field is read)
    double gscale;
    int store_bf16;                  // 1: round every stored Y / ACC value to bfloat16 (RN)
    // FP32 copies of cx .. cax, filled by the FP32 TMA launcher (the kernel reads them from
    // the parameter bank instead of holding converted values in registers)
    float fcx, fch, fcu, fck, fca, fcau, fcak, fcay, fcax;
};

// Arguments of the pointwise kernel (kernels_aux.cu).
struct PointArgs {
    int mode;        // 0: |q1|^2 (norm); 1: MGS pass; 2: Krylov combine; 3: copy; 4: swap;
                     // 5: <q_{j+1}, q_k> after a matrix-vector product (flat); 6: zero the
                     // fields fmask of vector dst; 7: |slot j+1|^2 into kry[KRY_AN] (flat);
                     // 8: multi-output Krylov combine (flat)
    int j, k, m;
    int src, dst;    // copy / swap vectors; combine: destination vector (mode 2)
    int notail;      // mode 0: 1 = start an Arnoldi process without the augmented tail;
                     // 2 = start from the tail already in slot 1 (adaptive substeps)
    int fmask;       // fields for copy / swap (bit f)
    double tol;
    double* partials;
    unsigned int* counters;
    void* out;             // combine (mode 2): when set, problem p's result goes to the
    long long out_stride;  // caller's buffer at out + p * out_stride elements, not vector dst
    // multi-output combine (mode 8): nout outputs from one read of the basis, output q with the
    // coefficients ecoef[(p (nout + final) + q) MAX_M ..] going to out + q out_qstride +
    // p out_stride (out set) or to vector dst + q; with final = 1 one more output, the last
    // coefficient row, goes to vector 0 (the state; every element is read before it is written)
    int nout, final_out;
    const double* ecoef;
    long long out_qstride;
};

// Host-side launchers (defined in kernels_stencil.cu / kernels_aux.cu).
int upload_stencil_tables(int order, const double* fs_uyy, const double* fs_uy,
                          const double* fs_dwy);
void launch_stage(int precision, int R, int nblocks, const ProblemDev* probs,
                  const int* tile_prob, const StageArgs& a, cudaStream_t s);
void launch_leapfrog(int precision, int R, int nblocks, const ProblemDev* probs,
                     const int* tile_prob, int cur, int prev, int variant, double dt,
                     cudaStream_t s);
// Pointwise parts of the leap-frog adjoint step (mode 0: q from lambda; mode 1: lambda update
// from y = H^T q); a1_base: the second cotangent vector of every shot (lam of w^{n-1}).
void launch_leapfrog_adjoint(int precision, int nblocks, const ProblemDev* probs, const int* tile_prob,
                             int mode, int qv, int yv, void* a1_base, double dt, cudaStream_t s);

// kernels_3d.cu: three-dimensional forward pass and leap-frog step.
int upload_stencil_tables_3d(const double* fs_uzz, const double* fs_uz, const double* fs_dwz);
void launch_stage3d(int precision, int R, int nblocks, const ProblemDev* probs,
                    const int* tile_prob, const StageArgs& a, cudaStream_t s);
void launch_leapfrog3d(int precision, int R, int nblocks, const ProblemDev* probs,
                       const int* tile_prob, int cur, int prev, int variant, double dt,
                       cudaStream_t s);

// kernels_tma3d.cu: persistent TMA-fed FP32 forward pass of three-dimensional problems.
int upload_tma3d_tables(const double* fs_uzz, const double* fs_uz, const double* fs_dwz);
int tma3d_tasks_of(const ProblemDev& P);
int build_tensor_maps3d(std::vector<ProblemDev>& probs, int R, const std::vector<int>& work_vecs,
                        void** d_maps_inout);
int launch_stage_tma3d(int R, int warps, const ProblemDev* probs, const int* tbase, int nprob,
                       int ntasks, const StageArgs& a, int* err, cudaStream_t s);
int launch_leapfrog_tma3d(int R, int warps, const ProblemDev* probs, const int* tbase, int nprob,
                          int ntasks, int cur, int prev, int variant, double dt, int* err,
                          cudaStream_t s);

// kernels_tma.cu: persistent TMA-fed FP32 forward pass.
int upload_tma_tables(const double* fs_uyy, const double* fs_uy, const double* fs_dwy);
int build_tensor_maps(std::vector<ProblemDev>& probs, int R, const std::vector<int>& work_vecs,
                      void** d_maps_inout);
constexpr int TMA_NUM_VARIANTS = 15;
// One 2D FP32 leap-frog step through the persistent TMA pass (column-pair consumers on
// 64 x 30 tiles); tbase and ntiles are those of the 30-row map set.
int launch_leapfrog_tma(int R, const ProblemDev* probs, const int* tbase, int nprob, int ntiles, int cur,
                        int prev, int variant, double dt, int* err, cudaStream_t s);
// The FWI gradient pass through the persistent TMA pass (column-pair consumers on 64 x 30
// tiles, the 30-row map set).
int launch_grad_tma(int R, const ProblemDev* probs, const int* tbase, int nprob, int ntiles,
                    const StageArgs& a, int* err, cudaStream_t s);
// The transposed pass H^T through the persistent TMA pipeline (FP32, no dot partner, no
// gradient; 64 x 18 tiles, the 18-row map set).
int launch_transpose_tma(int R, const ProblemDev* probs, const int* tbase, int nprob, int ntiles,
                         const StageArgs& a, int* err, cudaStream_t s);
int launch_stage_tma(int variant, int R, const ProblemDev* probs, const int* tbase, int nprob,
                     int ntiles, const StageArgs& a, int* err, cudaStream_t s);
int tma_variant_tile_height(int v);
// Tile height of variant v for a pass that does (reads_a) or does not read an A operand
// (composite variants pick their tile by it).
int tma_variant_tile_height_for(int v, bool reads_a);
// Tile heights of the 2D TMA map sets (set k has tile height TMA_SET_HEIGHTS[k]).
constexpr int TMA_NUM_SETS = 8;
constexpr int TMA_SET_HEIGHTS[TMA_NUM_SETS] = {16, 8, 20, 18, 24, 36, 28, 30};
int tma_map_set(int tile_height);
void tma_variant_describe(int v, int* by, int* nw, int* nst);

void launch_set_clock(const ProblemDev* probs, int nprob, double t, double dt, cudaStream_t s);
void launch_reset_cursor(const ProblemDev* probs, int nprob, cudaStream_t s);
void launch_prologue(const ProblemDev* probs, int nprob, int kind, int m, double gamma,
                     double c0, double c1, cudaStream_t s);
void launch_record(int precision, const ProblemDev* probs, int nprob, int vec, cudaStream_t s);
void launch_point(int precision, int nblocks, const ProblemDev* probs, const int* tile_prob,
                  const PointArgs& pa, cudaStream_t s);
// Flat pointwise passes (modes 0, 1, 2 of PointArgs) over whole padded vectors, PCHUNK
// elements per block; pbase: nprob + 1 prefix sums of the problems' chunk counts, then, from
// int offset flat_block_table(nprob), one (problem, chunk within the problem) pair per block.
__host__ __device__ constexpr int flat_block_table(int nprob) { return (nprob + 2) & ~1; }
void launch_point_flat(int precision, int nchunks, const ProblemDev* probs, const int* pbase,
                       int nprob, const PointArgs& pa, cudaStream_t s);
// Non-finite check of every problem's state vector (and its Arnoldi flag): sets bit 2 of *err.
void launch_nonfinite_scan(int precision, int nchunks, const ProblemDev* probs, const int* pbase,
                           int nprob, int* err, cudaStream_t s);
// Pipeline-wait limit of the 2D TMA pass in ns (default 1 s) on the current device.
int set_tma_wait_limit_ns(unsigned long long ns);
void launch_inject(int precision, void* adj, long long vec_elems, const void* values,
                   const int* rec_off, const int* nrec, int nshots, int max_rec, cudaStream_t s);
void launch_sum_shots(int precision, const void* in, void* out, long long n, int nshots,
                      cudaStream_t s);
int launch_expm(const ProblemDev* probs, int nprob, int mmax, cudaStream_t s, double hscale = 1.0);
// exp(tau_q H_meff) e_1 for ntau (<= MAX_TAU) values of tau in one launch, into
// out[(p ntau + q) MAX_M ..] (the coefficients of a multi-output Krylov combine, mode 8)
constexpr int MAX_TAU = 5;
struct ExpmTaus {
    int n;
    double tau[MAX_TAU];
    double* out;
};
int launch_expm_multi(const ProblemDev* probs, int nprob, int mmax, cudaStream_t s, const double* taus, int ntau,
                      double* out);

// kernels_mgs.cu: the modified Gram-Schmidt steps of one Arnoldi column (first dot, then
// k = k0 .. kmax) in one cooperative launch over the flat chunks, q_{j+1} in shared memory.
constexpr int MGS_MAX_CPB = 4;   // chunks per block at most
struct MgsArgs {
    int j, k0, kmax, m, cpb;
    double tol;
    double* partials;     // 2 x nchunks
    unsigned int* bar;    // [2]: grid-barrier arrivals and generation
    int* err;             // error word (bit 0: a barrier wait gave up)
};
// Chunks per block for which the grid is co-resident (smallest), or 0 if none is.
int mgs_column_chunks_per_block(int precision, int nchunks);
int launch_mgs_column(int precision, int nchunks, int cpb, const ProblemDev* probs, const int* pbase, int nprob,
                      const MgsArgs& ma, cudaStream_t s);
int set_mgs_wait_limit_ns(unsigned long long ns);
void launch_faber_coeffs(double dt, double gamma, double c0, double c1, int m, double* out,
                         cudaStream_t s);

}  // namespace ewv
