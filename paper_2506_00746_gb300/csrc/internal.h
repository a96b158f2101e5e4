// internal.h -- context, kernel parameter blocks and the per-(dim, order) dispatch table of the
// FEOD library.  Not part of the public ABI (include/feod.h is).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/feod.h"
#include "dfloat.cuh"

namespace feod {

constexpr int MAXQ = 7;                 // points per direction: order 6 -> 7 nodes / Gauss points
constexpr int MAX_ORDER = 6;

// Largest tile edge (elements per CTA = tile^dim) per (dim, order); also the default.  The
// element kernels are compiled with launch bounds for this many elements per CTA, so a context
// may use this tile or a smaller one.  3D order 6 takes one-element tiles: a 2x2x2 tile of order 6
// needs about 134 KB of shared memory in the FP32 tile kernel (one CTA per SM), a one-element tile
// about 18 KB.
constexpr int max_tile(int dim, int order)
{
    return dim == 3 ? (order == 1 ? 4 : order == 2 ? 3 : order <= 5 ? 2 : 1) : (order <= 3 ? 8 : 6);
}
constexpr int max_threads(int dim, int order)
{
    return dim == 3 ? max_tile(3, order) * max_tile(3, order) * max_tile(3, order) * (order + 1) * (order + 1)
                    : max_tile(2, order) * max_tile(2, order) * (order + 1);
}

// Slot code of a tile slot: bits 0..29 global DOF, bit 30 essential, bit 31 halo (the slot's DOF
// is owned by a neighbouring tile; this tile's partial sum goes to the halo buffer).
constexpr uint32_t SLOT_GMASK = 0x3FFFFFFFu;
constexpr uint32_t SLOT_ESS = 0x40000000u;
constexpr uint32_t SLOT_HALO = 0x80000000u;
constexpr uint32_t SLOT_INVALID = 0xFFFFFFFFu;
constexpr int64_t MAX_DOFS = (int64_t)SLOT_GMASK;   // 2^30 - 1

// Packed coefficient pairs of the double-float stages (empty for other types).  Each table pairs
// the rows i, i + 1 of a matrix M at column k, entry [(i / 2) MAXQ + k] (an odd last row with 0):
//   Bq:  M = B        (interpolation, i < Q1, k < D1)
//   Bt:  M = B^T      (transposed interpolation, i < D1, k < Q1)
//   Dq:  M = Dc       (collocation derivative, i, k < Q1)
//   Dt:  M = Dc^T
constexpr int NPK = (MAXQ + 1) / 2 * MAXQ;
template <typename T>
struct DfPairsT {};
template <>
struct DfPairsT<dfloat> {
    df2c Bq[NPK], Bt[NPK], Dq[NPK], Dt[NPK];
};

// 1D basis tables on the reference interval [0,1], row-major [q][a] with q < Q1, a < D1:
// B = phi_a(xi_q), G = phi_a'(xi_q), and the products used by the Jacobi diagonal.
template <typename T>
struct BasisT {
    T B[MAXQ * MAXQ];
    T G[MAXQ * MAXQ];
    T B2[MAXQ * MAXQ];   // B^2
    T G2[MAXQ * MAXQ];   // G^2
    T BG[MAXQ * MAXQ];   // B*G
    T Dc[MAXQ * MAXQ];   // collocation derivative at the Gauss points: Dc[q][j] = l_j'(x_q)
    DfPairsT<T> pk;
};

// FP32 1D basis tables as pairs, for packed (two-lane) FP32 multiply-adds: BG = (B, G),
// GB = (G, B), BB = (B, B), row-major [q][a].
struct BasisPairs {
    float2 BG[MAXQ * MAXQ];
    float2 GB[MAXQ * MAXQ];
    float2 BB[MAXQ * MAXQ];
};

// Pointwise law kinds (uniform for a launch): kappa(base) = base^a with a = (p-2)/2.
enum LawKind : int { LAW_GENERIC = 0, LAW_P2 = 1, LAW_P3 = 2, LAW_P4 = 3 };

// Everything the element kernels need about the mesh, tiling and law.
struct OpParams {
    int n[3];         // elements per direction (x, y, z; 1 beyond dim)
    int T;            // tile edge in elements
    int nt[3];        // tiles per direction
    int S;            // slots per tile = (k T + 1)^dim
    int SE;           // slots per tile edge = k T + 1
    int Spad;         // per-tile stride of slot codes and halo entries (S rounded up to 4)
    int law;          // LawKind
    int64_t ntiles;
    int64_t t0;       // first tile of a launch (the tile kernels take one tile per CTA from t0)
    int64_t tqs32;    // per-tile stride (floats) of the FP32 tangent, a multiple of 4
    int64_t tqs64;    // per-tile stride (doubles) of the FP64 tangent, a multiple of 2
    const uint32_t *slot;   // [ntiles][Spad]
    const uint32_t *hdst;   // [ntiles][Spad]: position of a halo slot's partial sum in the halo array
    const uint16_t *gt_off; // in-tile G^T table: slot s sums Ye[gt_src[j]], j in [gt_off[s], gt_off[s+1])
    const uint16_t *gt_src; // (same for every tile; padded elements contribute exact zeros)
    int *err;               // device error word (bounded waits that time out set it)
    const double *geo;      // [nepad][NG][NQ]
    const double *kr;       // [nepad] kappa_rho per element (internal order) or nullptr
    const double *dkr;      // [nepad] kappa_rho' per element or nullptr
    const int *skip;        // if non-null and *skip != 0 the kernel returns at once (CG batches)
    double law_a;     // (p-2)/2
    double eps2;      // eps^2
};

// Fix-up (deterministic G^T across tiles): y[fix_g[r]] += row r's halo entries, the partial sums
// of the non-owning tiles, stored contiguously in ascending tile order.  A DOF on m interior tile
// planes has 2^m - 1 non-owning tiles, so the rows come in runs by length: n1 rows of 1 entry (a
// tile face), then n3 rows of 3 (a tile edge), then the rest of 7 (a tile corner), each run
// sorted by DOF; a row's first entry follows from its number (fix_entries), so no offset table
// is read.
struct FixParams {
    int64_t nfix, n1, n3;
    int64_t r0, r1;           // the rows a launch handles, [r0, r1) ([0, nfix) for the whole sum)
    const uint32_t *fix_g;
    const int *skip;
};

__host__ __device__ inline void fix_entries(const FixParams &F, int64_t r, uint32_t &first, uint32_t &count)
{
    if (r < F.n1) { first = (uint32_t)r; count = 1u; }
    else if (r < F.n1 + F.n3) { first = (uint32_t)(F.n1 + 3 * (r - F.n1)); count = 3u; }
    else { first = (uint32_t)(F.n1 + 3 * F.n3 + 7 * (r - F.n1 - F.n3)); count = 7u; }
}

// Geometry setup parameters.
struct GeomParams {
    int dim, d1, q1, T;
    int n[3], nt[3];               // elements and tiles per direction (1 beyond dim)
    int64_t nepad;
    double xq[MAXQ], wq[MAXQ];     // Gauss points / weights on [0,1]
    double xn[MAXQ];               // GLL nodes on [0,1]
    int f_kind;
    double f_const;
    double p;
};

// Launchers of one (dim, order) instantiation.  Each runs the element kernel and, where the
// kernel assembles a global vector, the halo fix-up, on `st`.
struct OpTable {
    int dim, d1;
    // residual (want_r) and/or quadrature-point tangent (T64 / T32 non-null) of u
    void (*residual)(fe_ctx *c, const double *u, double *r, double *T64, float *T32, cudaStream_t st);
    // partially assembled J v
    void (*jv_pa_64)(fe_ctx *c, const double *v, double *y, cudaStream_t st);
    void (*jv_pa_32)(fe_ctx *c, const float *v, float *y, cudaStream_t st);
    void (*jv_pa_32d)(fe_ctx *c, const double *v, double *y, cudaStream_t st);
    // double-float operator (FP32 word pairs) with FP64 vectors, from the double-float tangent
    void (*jv_pa_df)(fe_ctx *c, const double *v, double *y, cudaStream_t st);
    // stateless J(u) v with one dual direction
    void (*jv_dual_64)(fe_ctx *c, const double *u, const double *v, double *y, cudaStream_t st);
    void (*jv_dual_32)(fe_ctx *c, const double *u, const float *v, float *y, cudaStream_t st);
    void (*jv_dual_32d)(fe_ctx *c, const double *u, const double *v, double *y, cudaStream_t st);
    // Jacobi diagonal from the stored tangent
    void (*diag_64)(fe_ctx *c, double *d, cudaStream_t st);
    void (*diag_32)(fe_ctx *c, double *d, cudaStream_t st);
    // adjoint design gradient
    void (*vjp)(fe_ctx *c, const double *u, const double *lam, double *grad, cudaStream_t st);
    // raise the dynamic shared-memory limit of every kernel for this context's tile size
    // (called once at setup, so that no attribute call happens inside a graph capture)
    cudaError_t (*prepare)(fe_ctx *c);
    // bytes of dynamic shared memory of the largest kernel for tile size T
    size_t (*max_smem)(int S, int T);
    // the cached J v in pieces (3D tile kernels only): the tile kernel on tiles [t0, t0 + nt),
    // then the fix-up of rows [r0, r1); precision as fe_jacobian_action's (64, 48, 32, -32);
    // plain stream order (no programmatic launch)
    void (*jv_tiles)(fe_ctx *c, int precision, const void *v, void *y, int64_t t0, int64_t nt, cudaStream_t st);
    void (*fix_rows)(fe_ctx *c, int precision, void *y, int64_t r0, int64_t r1, cudaStream_t st);
    // the CG's FP32 operator with FP64 vectors (precision -32) fed by the FP32 rounding p32 of the
    // direction p (the CG direction kernel writes both): q = J p in FP64, bit for bit jv_pa_32d on
    // p; false, with nothing launched, where the tile kernel does not run
    bool (*jv_pa_32s)(fe_ctx *c, const float *p32, const double *p, double *q, cudaStream_t st);
};

const OpTable *find_ops(int dim, int d1);

}  // namespace feod

// The context.  Owns all device memory it allocates.
struct fe_ctx {
    int dim = 0, k = 0, d1 = 0, q1 = 0;
    int n[3] = { 1, 1, 1 };                     // elements per direction (1 beyond dim)
    int natural = 0;                            // mask of box faces whose DOFs are not essential
    int T = 0, S = 0, SE = 0, NE = 0;           // tiling
    int nt[3] = { 1, 1, 1 };                    // tiles per direction
    int Spad = 0;                               // per-tile slot stride
    int64_t tqs32 = 0, tqs64 = 0;               // per-tile tangent strides (elements)
    uint16_t *d_gt_off = nullptr, *d_gt_src = nullptr;   // in-tile G^T table
    // grid (= number of tiles) of the tile-level 3D J v kernel per variant [FP64, FP32, FP32 with
    // FP64 vectors, double-float with FP64 vectors]; 0 = that variant runs the per-element kernel
    int pipe_grid[4] = { 0, 0, 0, 0 };
    bool per_element = false;       // the cached J v uses the per-element kernel (comparison)
    bool res_tile = false;          // R(u) and the tangent run the tile-level kernel (3D)
    bool cg_shadow = false;         // the precision -32 CG feeds its operator an FP32 copy of p
    int smem_optin = 0;
    int *h_err = nullptr;                       // pinned mirror of d_err
    int NQ = 0, NS = 0, NG = 0;                 // points per element, sym entries, geo comps
    int64_t nl = 0, nfree = 0, ne = 0, nepad = 0, ntiles = 0;
    int device = 0;
    int num_sms = 0;

    // problem
    double p = 3.0, eps = 0.0, kappa_eps = 0.0, kappa_q = 1.0, f_const = 0.0;
    int f_kind = 0, law = 0;
    bool has_rho = false;

    // device arrays
    uint32_t *d_slot = nullptr;
    uint32_t *d_fix_g = nullptr, *d_hdst = nullptr;
    int64_t nfix = 0, nfixh = 0;
    double *d_vert = nullptr;
    double *d_geo = nullptr;
    double *d_rho = nullptr;      // public order
    double *d_kr = nullptr, *d_dkr = nullptr;   // internal order
    double *d_T64 = nullptr;
    float *d_T32 = nullptr;
    feod::dfloat *d_Tdf = nullptr;  // double-float copy of the FP64 tangent (allocated on first use)
    double *d_diag = nullptr;
    void *d_halo = nullptr;       // nfixh * 8 bytes: cross-tile partial sums in fix-up order
    int *d_err = nullptr;
    bool lin64 = false, lin32 = false, have_diag = false;
    bool lindf = false;           // d_Tdf holds the current FP64 tangent

    // Newton / CG work space (allocated on first use)
    double *w_r = nullptr, *w_d = nullptr, *w_trial = nullptr;
    float *w_dinv = nullptr;      // Jacobi scaling 1/diag(J), FP32
    double *w_dinv64 = nullptr;   // the same values in FP64 (the FP64 CG kernels' operand)
    double *w_cx = nullptr, *w_cr = nullptr, *w_cp = nullptr, *w_cq = nullptr;   // FP64 CG
    double *w_cz = nullptr;       // FP64 CG: the preconditioned residual dinv r
    float *w_fx = nullptr, *w_fr = nullptr, *w_fp = nullptr, *w_fq = nullptr;    // FP32 CG
    void *w_state = nullptr;      // device CG state
    double *w_partial = nullptr;  // reduction partials
    void *h_state = nullptr;      // pinned host mirror
    cudaStream_t own_stream = nullptr;
    // fe_jacobian_action_host in z-chunks: copy streams, events, the fix-up rows' DOFs on the host
    bool chunked_host = true;
    cudaStream_t cp_in = nullptr, cp_out = nullptr;
    cudaStream_t cp_tile[2] = { nullptr, nullptr };   // the chunks' tile kernels, alternately
    cudaStream_t cp_fix = nullptr;                    // the chunks' fix-ups (high priority)
    cudaEvent_t chunk_ev[17] = {};
    cudaEvent_t tile_ev[8] = {};
    std::vector<uint32_t> h_fix_g;
    // captured CG batches: [0] FP64 operator and vectors, [1] FP32 operator with FP64 vectors,
    // [2] FP32 operator and vectors, [3] double-float operator with FP64 vectors
    cudaGraphExec_t cg_exec[4] = { nullptr, nullptr, nullptr, nullptr };
    int cg_batch[4] = { 0, 0, 0, 0 };
    int64_t cg_launches[4] = { 0, 0, 0, 0 };
    // the device-side CG loop per precision: one conditional WHILE node around cg_loop_m iterations
    cudaGraphExec_t cg_loop_exec[4] = { nullptr, nullptr, nullptr, nullptr };
    int cg_loop_m[4] = { 0, 0, 0, 0 };

    feod::OpParams op{};
    feod::FixParams fix{};
    feod::BasisT<double> b64{};
    feod::BasisT<float> b32{};
    feod::BasisT<feod::dfloat> bdf{};
    feod::BasisPairs p32{};
    feod::GeomParams gp{};
    const feod::OpTable *ops = nullptr;

    // profiling / counting
    bool prof = false;
    bool capturing = false;       // inside one of the library's own CG graph captures
    int64_t launches = 0;
    struct ProfRec { int name; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    std::vector<std::string> prof_names;
    std::vector<int64_t> prof_count;
    std::vector<double> prof_ms;

    int64_t mem_bytes = 0;
    std::string err;
};

namespace feod {

// Library-internal calls on one context (implemented in api.cu), used by the batch runtime.
// residual_tangent32: R(u) into r (nullptr: none) and the FP32 quadrature-point tangent at u,
// fused; jacobi_diag32: diag(J) from the stored FP32 tangent.  Both stream-ordered on st.
fe_status residual_tangent32(fe_ctx *c, const double *u, double *r, cudaStream_t st);
fe_status jacobi_diag32(fe_ctx *c, double *d, cudaStream_t st);
fe_status set_error(fe_ctx *c, fe_status s, const char *msg);
// alloc_tangent32: the (zero-filled) FP32 tangent storage, without computing it
fe_status alloc_tangent32(fe_ctx *c);

// Profiling bracket around one kernel launch.
int prof_name_id(fe_ctx *c, const char *name);
void prof_begin(fe_ctx *c, int name_id, cudaStream_t st, cudaEvent_t *a);
void prof_end(fe_ctx *c, int name_id, cudaStream_t st, cudaEvent_t a);

struct LaunchScope {
    fe_ctx *c; int id; cudaStream_t st; cudaEvent_t a = nullptr;
    LaunchScope(fe_ctx *c_, const char *name, cudaStream_t st_) : c(c_), st(st_) {
        c->launches++;
        id = c->prof ? prof_name_id(c, name) : -1;
        if (c->prof) prof_begin(c, id, st, &a);
    }
    ~LaunchScope() { if (c->prof) prof_end(c, id, st, a); }
};

}  // namespace feod
