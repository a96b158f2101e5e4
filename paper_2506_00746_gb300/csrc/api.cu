// api.cu -- the C ABI of include/feod.h: context setup (explicit G index arrays, basis tables,
// geometry), operator calls, the Jacobi-preconditioned CG and the Newton-CG driver.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"
#include "vector_kernels.h"

namespace feod {
void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &w);
void gll_nodes(int k, std::vector<double> &x);
void lagrange_tables(const std::vector<double> &nodes, const std::vector<double> &pts, std::vector<double> &val,
                     std::vector<double> &der);

// instantiation units (inst_*.cu)
const OpTable *ops_2d(int d1);
const OpTable *ops_3d_1();
const OpTable *ops_3d_2();
const OpTable *ops_3d_3();
const OpTable *ops_3d_4();
const OpTable *ops_3d_5();
const OpTable *ops_3d_6();

const OpTable *find_ops(int dim, int d1)
{
    if (dim == 2) return ops_2d(d1);
    switch (d1) {
    case 2: return ops_3d_1();
    case 3: return ops_3d_2();
    case 4: return ops_3d_3();
    case 5: return ops_3d_4();
    case 6: return ops_3d_5();
    case 7: return ops_3d_6();
    default: return nullptr;
    }
}

// ------------------------------------------------------------------------------------------------
// profiling
// ------------------------------------------------------------------------------------------------
int prof_name_id(fe_ctx *c, const char *name)
{
    for (size_t i = 0; i < c->prof_names.size(); ++i)
        if (c->prof_names[i] == name) return (int)i;
    c->prof_names.emplace_back(name);
    c->prof_count.push_back(0);
    c->prof_ms.push_back(0.0);
    return (int)c->prof_names.size() - 1;
}

static cudaEvent_t take_event(fe_ctx *c)
{
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(fe_ctx *c, int, cudaStream_t st, cudaEvent_t *a)
{
    *a = take_event(c);
    cudaEventRecord(*a, st);
}

void prof_end(fe_ctx *c, int id, cudaStream_t st, cudaEvent_t a)
{
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, st);
    c->prof_recs.push_back({ id, a, b });
}

}  // namespace feod

using namespace feod;

// ------------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------------
namespace {

fe_status fail(fe_ctx *c, fe_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
fe_status fail(fe_ctx *c, fe_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(c, e_ == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA, "%s: %s (%s:%d)",   \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
    } while (0)

#define CKLAUNCH()                                                                                        \
    do {                                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                                              \
        if (e_ != cudaSuccess)                                                                            \
            return fail(c, FE_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                                        \
    } while (0)

template <typename T>
cudaError_t dalloc(fe_ctx *c, T **p, size_t count)
{
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) c->mem_bytes += (int64_t)bytes;
    return e;
}

int64_t ipow64(int64_t b, int e) { int64_t r = 1; while (e-- > 0) r *= b; return r; }

// default tile edge (elements per CTA = T^dim) per (dim, order): the largest the kernels support
int default_tile(int dim, int k) { return max_tile(dim, k); }

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

CgState *cg_state(fe_ctx *c) { return reinterpret_cast<CgState *>(c->w_state); }
CgState *cg_host(fe_ctx *c) { return reinterpret_cast<CgState *>(c->h_state); }

fe_status ensure_work(fe_ctx *c)
{
    if (c->w_r) return FE_OK;
    const size_t n = (size_t)c->nl;
    CK(dalloc(c, &c->w_r, n));
    CK(dalloc(c, &c->w_d, n));
    CK(dalloc(c, &c->w_trial, n));
    CK(dalloc(c, &c->w_dinv, n));
    CK(dalloc(c, &c->w_dinv64, n));
    CK(dalloc(c, &c->w_cx, n));
    CK(dalloc(c, &c->w_cr, n));
    CK(dalloc(c, &c->w_cp, n));
    CK(dalloc(c, &c->w_cq, n));
    CK(dalloc(c, &c->w_cz, n));
    CK(dalloc(c, &c->w_fx, n));
    CK(dalloc(c, &c->w_fr, n));
    CK(dalloc(c, &c->w_fp, n));
    CK(dalloc(c, &c->w_fq, n));
    CgState *s = nullptr;
    CK(dalloc(c, &s, 2));
    CK(cudaMemset(s, 0, 2 * sizeof(CgState)));
    c->w_state = s;
    CK(dalloc(c, &c->w_partial, 3 * RED_BLOCKS));
    CK(cudaMallocHost(&c->h_state, 2 * sizeof(CgState)));
    CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    return FE_OK;
}

fe_status ensure_tangent(fe_ctx *c, bool f64, bool f32)
{
    // zero-filled: padded elements of ragged tiles keep a zero tangent, so they add exact zeros
    const size_t n64 = (size_t)c->ntiles * c->tqs64, n32 = (size_t)c->ntiles * c->tqs32;
    if (f64 && !c->d_T64) { CK(dalloc(c, &c->d_T64, n64)); CK(cudaMemset(c->d_T64, 0, n64 * sizeof(double))); }
    if (f32 && !c->d_T32) { CK(dalloc(c, &c->d_T32, n32)); CK(cudaMemset(c->d_T32, 0, n32 * sizeof(float))); }
    if (!c->d_diag) CK(dalloc(c, &c->d_diag, (size_t)c->nl));
    return FE_OK;
}

// The double-float tangent: allocated on first use, split from the FP64 tangent when that has
// changed since (stream-ordered on st).
fe_status prepare_tangent_df(fe_ctx *c, cudaStream_t st)
{
    if (c->lindf) return FE_OK;
    if (!c->lin64) return fail(c, FE_ERR_STATE, "no FP64 linearisation cached (call fe_linearize)");
    const size_t n64 = (size_t)c->ntiles * c->tqs64;
    if (!c->d_Tdf) CK(dalloc(c, &c->d_Tdf, n64));
    {
        LaunchScope ls(c, "split_df", st);
        k_split_df<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->d_T64, c->d_Tdf, (int64_t)n64);
    }
    CKLAUNCH();
    c->lindf = true;
    return FE_OK;
}

// deterministic dot product, synchronous on stream st
fe_status dot_sync(fe_ctx *c, const double *a, const double *b, double *out, cudaStream_t st)
{
    CgState *ds = cg_state(c) + 1;
    {
        LaunchScope ls(c, "dot", st);
        k_dot<<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, c->nl, c->w_partial + 2 * RED_BLOCKS, &ds->counter, &ds->scalar);
    }
    CKLAUNCH();
    CK(cudaMemcpyAsync(&cg_host(c)[1].scalar, &ds->scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out = cg_host(c)[1].scalar;
    return FE_OK;
}

fe_status apply_jv_cached(fe_ctx *c, const void *v, void *y, int precision, cudaStream_t st)
{
    if (precision == 64) {
        if (!c->lin64) return fail(c, FE_ERR_STATE, "no FP64 linearisation cached (call fe_linearize)");
        c->ops->jv_pa_64(c, (const double *)v, (double *)y, st);
    } else if (precision == 32) {
        if (!c->lin32) return fail(c, FE_ERR_STATE, "no FP32 linearisation cached (call fe_linearize)");
        c->ops->jv_pa_32(c, (const float *)v, (float *)y, st);
    } else if (precision == -32) {
        if (!c->lin32) return fail(c, FE_ERR_STATE, "no FP32 linearisation cached (call fe_linearize)");
        c->ops->jv_pa_32d(c, (const double *)v, (double *)y, st);
    } else if (precision == 48) {
        fe_status s = prepare_tangent_df(c, st);
        if (s != FE_OK) return s;
        c->ops->jv_pa_df(c, (const double *)v, (double *)y, st);
    } else {
        return fail(c, FE_ERR_ARG, "precision must be 64, 48, 32 or -32");
    }
    CKLAUNCH();
    return FE_OK;
}

// the precision -32 CG feeds its FP32 operator an FP32 copy of the direction (tile kernel only)
bool cg_shadow(const fe_ctx *c) { return c->cg_shadow && c->ops->jv_pa_32s != nullptr; }

// Enqueue `m` CG iterations (J p, alpha, update, direction); every kernel is a no-op once the
// device flag `done` is set.  precision 64: FP64 operator and vectors; 48: double-float operator,
// FP64 vectors; -32: FP32 operator, FP64 vectors; 32: FP32 operator and vectors (CG scalars and
// inner-product sums in FP64).
void enqueue_cg(fe_ctx *c, int m, int precision, cudaStream_t st)
{
    CgState *s = cg_state(c);
    const int64_t n = c->nl;
    c->op.skip = &s->done;
    c->fix.skip = &s->done;
    for (int i = 0; i < m; ++i) {
        if (precision != 32) {
            // precision -32 with the tile kernel: the operator reads the FP32 copy of p that the
            // direction kernel writes (the conversion moves out of the operator's gather)
            float *p32 = precision == -32 && cg_shadow(c) ? c->w_fp : nullptr;
            if (precision == 64) c->ops->jv_pa_64(c, c->w_cp, c->w_cq, st);
            else if (precision == 48) c->ops->jv_pa_df(c, c->w_cp, c->w_cq, st);
            else if (!p32) c->ops->jv_pa_32d(c, c->w_cp, c->w_cq, st);
            else c->ops->jv_pa_32s(c, p32, c->w_cp, c->w_cq, st);
            { LaunchScope ls(c, "cg_alpha", st); k_cg_alpha<<<RED_BLOCKS, RED_THREADS, 0, st>>>(c->w_cp, c->w_cq, n, s, c->w_partial); }
            { LaunchScope ls(c, "cg_update", st); k_cg_update<<<RED_BLOCKS, RED_THREADS, 0, st>>>(c->w_cr, c->w_cq, c->w_dinv64, c->w_cz, n, s, c->w_partial); }
            { LaunchScope ls(c, "cg_direction", st); k_cg_direction<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_cx, c->w_cp, p32, c->w_cz, c->w_cr, n, s, c->w_partial); }
        } else {
            c->ops->jv_pa_32(c, c->w_fp, c->w_fq, st);
            { LaunchScope ls(c, "cg_alpha32", st); k_cg_alpha32<<<RED_BLOCKS, RED_THREADS, 0, st>>>(c->w_fp, c->w_fq, n, s, c->w_partial); }
            { LaunchScope ls(c, "cg_update32", st); k_cg_update32<<<RED_BLOCKS, RED_THREADS, 0, st>>>(c->w_fx, c->w_fr, c->w_fp, c->w_fq, c->w_dinv, n, s, c->w_partial); }
            { LaunchScope ls(c, "cg_direction32", st); k_cg_direction32<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_fp, c->w_fr, c->w_dinv, n, s); }
        }
    }
    c->op.skip = nullptr;
    c->fix.skip = nullptr;
}

// The device error word: a kernel whose bounded wait timed out has set it.  Synchronises st; on
// an error resets the word and reports.
fe_status check_device_error(fe_ctx *c, cudaStream_t st)
{
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr == 0) return FE_OK;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return fail(c, FE_ERR_CUDA, "a kernel's bounded wait timed out (code %d); results of that call are invalid", herr);
}

// CG on J x = b (x from 0) with the cached linearisation and preconditioner dinv, on c->own_stream.
fe_status run_cg(fe_ctx *c, const double *b, double rtol, int max_iter, int precision, int batch, int graph_mode,
                 int *iters, int *done_code)
{
    // graph_mode: 0 plain launches, 1 captured batches with a host check after each, 2 the whole
    // solve on the device (conditional WHILE node)
    const bool use_graph = graph_mode != 0, device_loop = graph_mode == 2;
    cudaStream_t st = c->own_stream;
    CgState *s = cg_state(c);
    if (precision == 48) {
        // solve for b / 2^e (2^e near the RMS of b), staged in q (first written by J p)
        CgState *ds = s + 1;
        {
            LaunchScope ls(c, "dot", st);
            k_dot<<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, b, c->nl, c->w_partial + 2 * RED_BLOCKS, &ds->counter,
                                                      &ds->scalar);
        }
        {
            LaunchScope ls(c, "scale_rhs", st);
            k_scale_rhs<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_cq, b, c->nl, &ds->scalar, s);
        }
        LaunchScope ls(c, "cg_init", st);
        k_cg_init<<<RED_BLOCKS, RED_THREADS, 0, st>>>(c->w_cq, c->w_dinv64, c->w_cx, c->w_cr, c->w_cp, nullptr,
                                                      c->nl, s, rtol, max_iter, c->w_partial);
    } else if (precision != 32) {
        LaunchScope ls(c, "cg_init", st);
        k_cg_init<<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, c->w_dinv64, c->w_cx, c->w_cr, c->w_cp,
                                                      precision == -32 && cg_shadow(c) ? c->w_fp : nullptr, c->nl,
                                                      s, rtol, max_iter, c->w_partial);
    } else {
        CgState *ds = s + 1;
        {
            LaunchScope ls(c, "dot", st);
            k_dot<<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, b, c->nl, c->w_partial + 2 * RED_BLOCKS, &ds->counter,
                                                      &ds->scalar);
        }
        LaunchScope ls(c, "cg_init32", st);
        k_cg_init32<<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, c->w_dinv, c->w_fx, c->w_fr, c->w_fp, c->nl, s,
                                                        &ds->scalar, rtol, max_iter, c->w_partial);
    }
    CKLAUNCH();
    if (batch < 1) batch = 1;
    const int gi = precision == 64 ? 0 : precision == -32 ? 1 : precision == 32 ? 2 : 3;
    if (use_graph && !device_loop && (c->cg_exec[gi] == nullptr || c->cg_batch[gi] != batch)) {
        if (c->cg_exec[gi]) { cudaGraphExecDestroy(c->cg_exec[gi]); c->cg_exec[gi] = nullptr; }
        const bool prof = c->prof;
        c->prof = false;
        const int64_t l0 = c->launches;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        enqueue_cg(c, batch, precision, st);
        c->capturing = false;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        c->prof = prof;
        if (e != cudaSuccess) return fail(c, FE_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        c->cg_launches[gi] = c->launches - l0;
        c->launches = l0;
        e = cudaGraphInstantiate(&c->cg_exec[gi], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(c, FE_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        c->cg_batch[gi] = batch;
    }
    CgState *h = cg_host(c);
    if (use_graph && device_loop) {
        // the whole solve as one graph launch: a conditional WHILE node whose body is `batch`
        // iterations and the condition kernel; no host round trip until the solve ends
        if (c->cg_loop_exec[gi] == nullptr || c->cg_loop_m[gi] != batch) {
            if (c->cg_loop_exec[gi]) { cudaGraphExecDestroy(c->cg_loop_exec[gi]); c->cg_loop_exec[gi] = nullptr; }
            cudaGraph_t g = nullptr;
            CK(cudaGraphCreate(&g, 0));
            cudaGraphConditionalHandle hc;
            cudaError_t e = cudaGraphConditionalHandleCreate(&hc, g, 1u, cudaGraphCondAssignDefault);
            cudaGraphNodeParams np = { cudaGraphNodeTypeConditional };   // aggregate: the rest zero
            np.conditional.handle = hc;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
            if (e == cudaSuccess) {
                cudaGraph_t body = np.conditional.phGraph_out[0];
                const bool prof = c->prof;
                c->prof = false;
                const int64_t l0 = c->launches;
                e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    c->capturing = true;
                    enqueue_cg(c, batch, precision, st);
                    c->capturing = false;
                    k_cg_continue<<<1, 1, 0, st>>>(hc, s);
                    e = cudaStreamEndCapture(st, &body);
                }
                c->prof = prof;
                c->cg_launches[gi] = c->launches - l0;
                c->launches = l0;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->cg_loop_exec[gi], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(c, FE_ERR_CUDA, "device CG loop graph: %s", cudaGetErrorString(e));
            c->cg_loop_m[gi] = batch;
        }
        CK(cudaGraphLaunch(c->cg_loop_exec[gi], st));
        CK(cudaMemcpyAsync(h, s, sizeof(CgState), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        // kernels run: `batch` iterations' launches (and the condition kernel) per body pass
        const int64_t passes = std::max<int64_t>(1, (h->iter + batch - 1) / batch);
        c->launches += passes * (c->cg_launches[gi] + 1);
    }
    for (; !(use_graph && device_loop);) {
        if (use_graph) {
            CK(cudaGraphLaunch(c->cg_exec[gi], st));
            c->launches += c->cg_launches[gi];
        } else {
            enqueue_cg(c, batch, precision, st);
            CKLAUNCH();
        }
        CK(cudaMemcpyAsync(h, s, sizeof(CgState), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (h->done) break;
    }
    {
        fe_status e = check_device_error(c, st);
        if (e != FE_OK) return e;
    }
    if (precision == 32) {
        // the FP32 solution, unscaled, into the FP64 solution vector
        LaunchScope ls(c, "cg_widen", st);
        k_cg_widen<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_cx, c->w_fx, c->nl, s);
    } else if (precision == 48) {
        LaunchScope ls(c, "unscale", st);
        k_unscale<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_cx, c->nl, s);
    }
    CKLAUNCH();
    if (iters) *iters = h->iter;
    if (done_code) *done_code = h->done;
    return FE_OK;
}

}  // namespace

namespace feod {
fe_status residual_tangent32(fe_ctx *c, const double *u, double *r, cudaStream_t st)
{
    fe_status s = ensure_tangent(c, false, true);
    if (s != FE_OK) return s;
    c->ops->residual(c, u, r, nullptr, c->d_T32, st);
    CKLAUNCH();
    c->lin32 = true;
    return FE_OK;
}

fe_status jacobi_diag32(fe_ctx *c, double *d, cudaStream_t st)
{
    if (!c->lin32) return fail(c, FE_ERR_STATE, "no FP32 linearisation");
    c->ops->diag_32(c, d, st);
    CKLAUNCH();
    return FE_OK;
}

fe_status set_error(fe_ctx *c, fe_status s, const char *msg) { return fail(c, s, "%s", msg); }

fe_status alloc_tangent32(fe_ctx *c) { return ensure_tangent(c, false, true); }
}  // namespace feod

// ------------------------------------------------------------------------------------------------
// setup
// ------------------------------------------------------------------------------------------------
extern "C" fe_status fe_setup(const fe_mesh *mesh, int order, int q1d, const fe_problem *prob, fe_ctx **out)
{
    return fe_setup_ex(mesh, order, q1d, prob, nullptr, out);
}

static fe_status setup_impl(fe_ctx *c, const fe_mesh *mesh, int order, const fe_problem *prob,
                            const fe_setup_opts *opts)
{
    const int dim = mesh->dim, k = order;
    c->dim = dim; c->k = k; c->d1 = k + 1; c->q1 = k + 1;
    for (int d = 0; d < 3; ++d) c->n[d] = d < dim ? mesh->n[d] : 1;
    c->natural = mesh->natural_faces & (dim == 3 ? 63 : 15);
    const int *n = c->n;
    c->NQ = (int)ipow64(c->q1, dim);
    c->NS = dim == 3 ? 6 : 3;
    c->NG = c->NS + 2;
    c->p = prob->p; c->eps = prob->eps; c->f_kind = prob->f_kind; c->f_const = prob->f_const;
    c->kappa_eps = prob->kappa_eps; c->kappa_q = prob->kappa_q;
    c->has_rho = prob->rho != nullptr;
    c->law = (prob->p == 2.0) ? LAW_P2 : (prob->p == 3.0) ? LAW_P3 : (prob->p == 4.0) ? LAW_P4 : LAW_GENERIC;
    // DOF lattice (k n_d + 1) per direction; a DOF is essential when it lies on a box face that
    // is not natural
    int64_t m[3] = { 1, 1, 1 }, mfree[3] = { 1, 1, 1 };
    for (int d = 0; d < dim; ++d) {
        m[d] = (int64_t)k * n[d] + 1;
        mfree[d] = m[d] - ((c->natural >> (2 * d)) & 1 ? 0 : 1) - ((c->natural >> (2 * d + 1)) & 1 ? 0 : 1);
    }
    c->nl = m[0] * m[1] * m[2];
    c->nfree = mfree[0] * mfree[1] * mfree[2];
    c->ne = (int64_t)n[0] * n[1] * n[2];
    if (c->nl > MAX_DOFS) return fail(c, FE_ERR_UNSUPPORTED, "%lld DOFs exceed the 2^30-1 limit", (long long)c->nl);

    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    int smem_optin = 0;
    CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    c->smem_optin = smem_optin;
    c->per_element = opts && opts->per_element;

    c->ops = find_ops(dim, c->d1);
    if (!c->ops) return fail(c, FE_ERR_UNSUPPORTED, "no kernels built for dim %d order %d", dim, k);

    // tile size
    int T = (opts && opts->tile > 0) ? opts->tile : default_tile(dim, k);
    if (T > max_tile(dim, k)) T = max_tile(dim, k);
    for (int d = 0; d < dim; ++d)
        if (T > n[d]) T = n[d];
    const int team = dim == 3 ? c->d1 * c->d1 : c->d1;
    for (;;) {
        const int NE = (int)ipow64(T, dim);
        const int S = (int)ipow64((int64_t)k * T + 1, dim);
        if (NE * team <= 1024 && c->ops->max_smem(S, T) <= (size_t)smem_optin) break;
        if (T == 1) return fail(c, FE_ERR_UNSUPPORTED, "order %d does not fit one element per CTA", k);
        --T;
    }
    c->T = T;
    c->NE = (int)ipow64(T, dim);
    for (int d = 0; d < 3; ++d) c->nt[d] = d < dim ? (n[d] + T - 1) / T : 1;
    c->ntiles = (int64_t)c->nt[0] * c->nt[1] * c->nt[2];
    c->nepad = c->ntiles * c->NE;
    c->SE = k * T + 1;
    c->S = (int)ipow64(c->SE, dim);
    c->Spad = (c->S + 3) & ~3;
    const int64_t tq_block = (int64_t)c->NE * c->NS * c->NQ;
    c->tqs32 = (tq_block + 3) & ~(int64_t)3;
    c->tqs64 = (tq_block + 1) & ~(int64_t)1;
    if ((double)c->ntiles * c->Spad >= 4294967295.0)
        return fail(c, FE_ERR_UNSUPPORTED, "tile slot index exceeds 32 bits");

    // --- in-tile G^T table: for every slot, the staged element outputs (el*NQ + local node) that
    //     sum into it, in ascending (z, y, x) element order; identical for every tile ---
    std::vector<uint16_t> gt_off(c->S + 1), gt_src;
    {
        gt_src.reserve((size_t)c->NE * c->NQ);
        for (int s = 0; s < c->S; ++s) {
            gt_off[s] = (uint16_t)gt_src.size();
            const int sc[3] = { s % c->SE, (s / c->SE) % c->SE, dim == 3 ? s / (c->SE * c->SE) : 0 };
            int ce[3][2], cl[3][2], cn[3];
            for (int d = 0; d < 3; ++d) {
                cn[d] = 0;
                if (d >= dim) { ce[d][0] = 0; cl[d][0] = 0; cn[d] = 1; continue; }
                for (int te = 0; te < T; ++te) {
                    const int a = sc[d] - k * te;
                    if (a >= 0 && a <= k) { ce[d][cn[d]] = te; cl[d][cn[d]] = a; cn[d]++; }
                }
            }
            for (int iz = 0; iz < cn[2]; ++iz)
                for (int iy = 0; iy < cn[1]; ++iy)
                    for (int ix = 0; ix < cn[0]; ++ix) {
                        const int el = ce[0][ix] + T * (ce[1][iy] + T * ce[2][iz]);
                        const int lo = cl[0][ix] + c->d1 * (cl[1][iy] + c->d1 * cl[2][iz]);
                        gt_src.push_back((uint16_t)(el * c->NQ + lo));
                    }
        }
        gt_off[c->S] = (uint16_t)gt_src.size();
        if (gt_src.size() != (size_t)c->NE * c->NQ || (size_t)c->NE * c->NQ > 65535)
            return fail(c, FE_ERR_UNSUPPORTED, "in-tile G^T table does not fit 16-bit indices");
    }

    // --- G as explicit index arrays: slot codes per tile, and the transposed halo index ---
    std::vector<uint32_t> slot((size_t)c->ntiles * c->Spad, SLOT_INVALID);
    std::vector<uint64_t> halo_pairs;   // (g << 32) | (t*S + s)
    for (int64_t t = 0; t < c->ntiles; ++t) {
        int64_t tc[3] = { 0, 0, 0 }, r = t;
        for (int d = 0; d < dim; ++d) { tc[d] = r % c->nt[d]; r /= c->nt[d]; }
        for (int s = 0; s < c->S; ++s) {
            int sc[3] = { s % c->SE, (s / c->SE) % c->SE, dim == 3 ? s / (c->SE * c->SE) : 0 };
            bool valid = true, ess = false, halo = false;
            int64_t gl[3] = { 0, 0, 0 };
            for (int d = 0; d < dim; ++d) {
                gl[d] = (int64_t)k * T * tc[d] + sc[d];
                if (gl[d] > (int64_t)k * n[d]) valid = false;
                if (gl[d] == 0 && !((c->natural >> (2 * d)) & 1)) ess = true;
                if (gl[d] == (int64_t)k * n[d] && !((c->natural >> (2 * d + 1)) & 1)) ess = true;
                if (sc[d] == k * T && tc[d] < c->nt[d] - 1) halo = true;
            }
            uint32_t code = SLOT_INVALID;
            if (valid) {
                const int64_t g = gl[0] + m[0] * (gl[1] + (dim == 3 ? m[1] * gl[2] : 0));
                code = (uint32_t)g | (ess ? SLOT_ESS : 0u) | (halo ? SLOT_HALO : 0u);
                if (halo && !ess) halo_pairs.push_back(((uint64_t)g << 32) | (uint64_t)(t * c->Spad + s));
            }
            slot[(size_t)t * c->Spad + s] = code;
        }
    }
    // The cross-tile partial sums are stored compactly in fix-up order: one row per DOF that
    // several tiles share, holding the non-owning tiles' partials in ascending tile order.  Rows
    // are grouped by their length (1, 3, 7: the DOF lies on 1, 2 or 3 interior tile planes), each
    // group sorted by DOF.  The partial of halo slot (t, s) goes to hdst[t][s], and the fix-up
    // adds row r to the owner's value y[fix_g[r]] in that order (fix_entries gives the row's
    // place).
    std::sort(halo_pairs.begin(), halo_pairs.end());
    std::vector<uint32_t> fix_g, hdst((size_t)c->ntiles * c->Spad, 0u);
    {
        std::vector<std::pair<size_t, size_t>> runs[3];      // [begin, end) in halo_pairs, by class
        for (size_t i = 0; i < halo_pairs.size();) {
            size_t j = i;
            while (j < halo_pairs.size() && (halo_pairs[j] >> 32) == (halo_pairs[i] >> 32)) ++j;
            const size_t cnt = j - i;
            const int cls = cnt == 1 ? 0 : cnt == 3 ? 1 : cnt == 7 ? 2 : -1;
            if (cls < 0) return fail(c, FE_ERR_UNSUPPORTED, "a DOF has %zu cross-tile partial sums", cnt);
            runs[cls].push_back({ i, j });
            i = j;
        }
        uint32_t pos = 0;
        for (int cls = 0; cls < 3; ++cls)
            for (const auto &rn : runs[cls]) {
                fix_g.push_back((uint32_t)(halo_pairs[rn.first] >> 32));
                for (size_t i = rn.first; i < rn.second; ++i) hdst[halo_pairs[i] & 0xFFFFFFFFu] = pos++;
            }
        c->fix.n1 = (int64_t)runs[0].size();
        c->fix.n3 = (int64_t)runs[1].size();
        c->nfixh = (int64_t)pos;
    }
    c->nfix = (int64_t)fix_g.size();

    // --- 1D rules and basis tables on [0,1] ---
    std::vector<double> gx, gw, nodes, val, der;
    gauss_legendre(c->q1, gx, gw);
    gll_nodes(k, nodes);
    std::vector<double> xq(c->q1), xn(c->d1);
    for (int q = 0; q < c->q1; ++q) { xq[q] = 0.5 * (gx[q] + 1.0); c->gp.xq[q] = xq[q]; c->gp.wq[q] = 0.5 * gw[q]; }
    for (int a = 0; a < c->d1; ++a) { xn[a] = 0.5 * (nodes[a] + 1.0); c->gp.xn[a] = xn[a]; }
    lagrange_tables(xn, xq, val, der);     // derivatives w.r.t. the [0,1] coordinate
    for (int q = 0; q < c->q1; ++q)
        for (int a = 0; a < c->d1; ++a) {
            const int i = q * c->d1 + a;
            const double B = val[i], G = der[i];
            c->b64.B[i] = B; c->b64.G[i] = G; c->b64.B2[i] = B * B; c->b64.G2[i] = G * G; c->b64.BG[i] = B * G;
            c->b32.B[i] = (float)B; c->b32.G[i] = (float)G; c->b32.B2[i] = (float)(B * B);
            c->b32.G2[i] = (float)(G * G); c->b32.BG[i] = (float)(B * G);
            c->p32.BG[i] = make_float2((float)B, (float)G);
            c->p32.GB[i] = make_float2((float)G, (float)B);
            c->p32.BB[i] = make_float2((float)B, (float)B);
            c->bdf.B[i] = dfloat(B); c->bdf.G[i] = dfloat(G); c->bdf.B2[i] = dfloat(B * B);
            c->bdf.G2[i] = dfloat(G * G); c->bdf.BG[i] = dfloat(B * G);
        }
    // collocation derivative: the Lagrange basis on the Gauss points, differentiated there
    std::vector<double> cval, cder;
    lagrange_tables(xq, xq, cval, cder);
    for (int i = 0; i < c->q1 * c->q1; ++i) {
        c->b64.Dc[i] = cder[i];
        c->b32.Dc[i] = (float)cder[i];
        c->bdf.Dc[i] = dfloat(cder[i]);
    }
    // packed double-float coefficient pairs (rows i, i + 1; an odd last row paired with 0)
    {
        const int d1 = c->d1, q1 = c->q1;
        const dfloat z(0);
        auto fill = [&](df2c *t, int ni, int nk, auto m) {
            for (int i = 0; i < ni; i += 2)
                for (int k = 0; k < nk; ++k)
                    t[(i / 2) * MAXQ + k] = df2c_pack(m(i, k), i + 1 < ni ? m(i + 1, k) : z);
        };
        fill(c->bdf.pk.Bq, q1, d1, [&](int i, int k) { return c->bdf.B[i * d1 + k]; });
        fill(c->bdf.pk.Bt, d1, q1, [&](int i, int k) { return c->bdf.B[k * d1 + i]; });
        fill(c->bdf.pk.Dq, q1, q1, [&](int i, int k) { return c->bdf.Dc[i * q1 + k]; });
        fill(c->bdf.pk.Dt, q1, q1, [&](int i, int k) { return c->bdf.Dc[k * q1 + i]; });
    }
    c->gp.dim = dim; c->gp.d1 = c->d1; c->gp.q1 = c->q1; c->gp.T = T;
    for (int d = 0; d < 3; ++d) { c->gp.n[d] = n[d]; c->gp.nt[d] = c->nt[d]; }
    c->gp.nepad = c->nepad; c->gp.f_kind = prob->f_kind; c->gp.f_const = prob->f_const; c->gp.p = prob->p;

    // --- device data ---
    const int64_t nvert = (int64_t)(n[0] + 1) * (n[1] + 1) * (dim == 3 ? n[2] + 1 : 1);
    CK(dalloc(c, &c->d_gt_off, gt_off.size()));
    CK(dalloc(c, &c->d_gt_src, gt_src.size()));
    CK(cudaMemcpy(c->d_gt_off, gt_off.data(), gt_off.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_gt_src, gt_src.data(), gt_src.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    CK(dalloc(c, &c->d_slot, slot.size()));
    CK(cudaMemcpy(c->d_slot, slot.data(), slot.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CK(dalloc(c, &c->d_fix_g, fix_g.size()));
    CK(dalloc(c, &c->d_hdst, hdst.size()));
    CK(cudaMemcpy(c->d_hdst, hdst.data(), hdst.size() * 4, cudaMemcpyHostToDevice));
    if (!fix_g.empty()) CK(cudaMemcpy(c->d_fix_g, fix_g.data(), fix_g.size() * 4, cudaMemcpyHostToDevice));
    CK(dalloc(c, &c->d_vert, (size_t)nvert * dim));
    CK(cudaMemcpy(c->d_vert, mesh->vertices, (size_t)nvert * dim * sizeof(double), cudaMemcpyHostToDevice));
    CK(dalloc(c, &c->d_geo, (size_t)c->nepad * c->NG * c->NQ));
    {
        double *h = nullptr;
        CK(dalloc(c, &h, (size_t)c->nfixh));
        c->d_halo = h;
    }
    CK(dalloc(c, &c->d_err, 1));
    CK(cudaMemset(c->d_err, 0, sizeof(int)));

    {
        const int64_t total = c->nepad * c->NQ;
        const int bs = 256;
        k_geometry<<<(unsigned)((total + bs - 1) / bs), bs>>>(c->gp, c->d_vert, c->d_geo, c->d_err);
        CKLAUNCH();
        c->launches++;
    }
    if (c->has_rho) {
        CK(dalloc(c, &c->d_rho, (size_t)c->ne));
        CK(cudaMemcpy(c->d_rho, prob->rho, (size_t)c->ne * sizeof(double), cudaMemcpyHostToDevice));
        CK(dalloc(c, &c->d_kr, (size_t)c->nepad));
        CK(dalloc(c, &c->d_dkr, (size_t)c->nepad));
        k_design_factors<<<(unsigned)((c->nepad + 255) / 256), 256>>>(c->gp, c->d_rho, c->kappa_eps, c->kappa_q,
                                                                       c->d_kr, c->d_dkr);
        CKLAUNCH();
        c->launches++;
    }
    int herr = 0;
    CK(cudaMemcpy(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return fail(c, FE_ERR_MESH, "det J <= 0 at a quadrature point (inverted or degenerate element)");

    // --- kernel parameter blocks ---
    for (int d = 0; d < 3; ++d) { c->op.n[d] = n[d]; c->op.nt[d] = c->nt[d]; }
    c->op.T = T; c->op.S = c->S; c->op.SE = c->SE; c->op.law = c->law;
    c->op.ntiles = c->ntiles; c->op.slot = c->d_slot; c->op.geo = c->d_geo;
    c->op.Spad = c->Spad; c->op.tqs32 = c->tqs32; c->op.tqs64 = c->tqs64;
    c->op.gt_off = c->d_gt_off; c->op.gt_src = c->d_gt_src; c->op.err = c->d_err;
    c->op.kr = c->d_kr; c->op.dkr = c->d_dkr; c->op.skip = nullptr;
    c->op.law_a = 0.5 * (prob->p - 2.0); c->op.eps2 = prob->eps * prob->eps;
    c->op.hdst = c->d_hdst;
    c->fix.nfix = c->nfix; c->fix.fix_g = c->d_fix_g;
    c->fix.r0 = 0; c->fix.r1 = c->nfix;
    c->fix.skip = nullptr;
    c->h_fix_g = std::move(fix_g);
    CK(c->ops->prepare(c));
    CK(cudaDeviceSynchronize());
    return FE_OK;
}

static thread_local std::string g_setup_error;

extern "C" fe_status fe_setup_ex(const fe_mesh *mesh, int order, int q1d, const fe_problem *prob,
                                 const fe_setup_opts *opts, fe_ctx **out)
{
    if (!out) return FE_ERR_ARG;
    *out = nullptr;
    g_setup_error.clear();
    if (!mesh || !prob || !mesh->vertices || (mesh->dim != 2 && mesh->dim != 3) || mesh->n[0] < 1 ||
        mesh->n[1] < 1 || (mesh->dim == 3 && mesh->n[2] < 1)) {
        g_setup_error = "invalid mesh or problem";
        return FE_ERR_ARG;
    }
    if (mesh->natural_faces < 0 || mesh->natural_faces > (mesh->dim == 3 ? 63 : 15)) {
        g_setup_error = "natural_faces must be a mask of the box faces (bits 0-5 in 3D, 0-3 in 2D)";
        return FE_ERR_ARG;
    }
    if (order < 1 || order > MAX_ORDER) { g_setup_error = "order must be 1..6"; return FE_ERR_UNSUPPORTED; }
    if (q1d != 0 && q1d != order + 1) { g_setup_error = "q1d must be 0 or order+1"; return FE_ERR_UNSUPPORTED; }
    if (!(prob->p >= 2.0 || (prob->p > 1.0 && prob->eps > 0.0)) || !(prob->eps >= 0.0)) {
        g_setup_error = "need p >= 2, or p > 1 with eps > 0";
        return FE_ERR_ARG;
    }
    if (prob->f_kind != 0 && prob->f_kind != 1) { g_setup_error = "f_kind must be 0 or 1"; return FE_ERR_ARG; }
    fe_ctx *c = new (std::nothrow) fe_ctx();
    if (!c) return FE_ERR_OOM;
    fe_status s = setup_impl(c, mesh, order, prob, opts);
    if (s != FE_OK) {
        g_setup_error = c->err;
        fe_destroy(c);
        return s;
    }
    *out = c;
    return FE_OK;
}

extern "C" void fe_destroy(fe_ctx *c)
{
    if (!c) return;
    void *ptrs[] = { c->d_gt_off, c->d_gt_src, c->d_slot, c->d_fix_g, c->d_hdst, c->d_vert, c->d_geo, c->d_rho, c->d_kr,
                     c->d_dkr, c->d_T64, c->d_T32, c->d_Tdf, c->d_diag, c->d_halo, c->d_err, c->w_r, c->w_d, c->w_trial,
                     c->w_dinv, c->w_dinv64, c->w_cx, c->w_cr, c->w_cp, c->w_cq, c->w_cz, c->w_fx, c->w_fr, c->w_fp, c->w_fq, c->w_state, c->w_partial };
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->cp_in) cudaStreamDestroy(c->cp_in);
    if (c->cp_out) cudaStreamDestroy(c->cp_out);
    if (c->cp_fix) cudaStreamDestroy(c->cp_fix);
    for (cudaStream_t t : c->cp_tile)
        if (t) cudaStreamDestroy(t);
    for (cudaEvent_t e : c->chunk_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->tile_ev)
        if (e) cudaEventDestroy(e);
    for (auto &g : c->cg_loop_exec)
        if (g) cudaGraphExecDestroy(g);
    for (auto &g : c->cg_exec)
        if (g) cudaGraphExecDestroy(g);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    for (auto &r : c->prof_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->prof_pool) cudaEventDestroy(e);
    delete c;
}

extern "C" const char *fe_last_error(const fe_ctx *c)
{
    if (!c) return g_setup_error.c_str();
    return c->err.c_str();
}

extern "C" const char *fe_status_string(fe_status s)
{
    switch (s) {
    case FE_OK: return "ok";
    case FE_ERR_ARG: return "invalid argument";
    case FE_ERR_MESH: return "invalid mesh (det J <= 0)";
    case FE_ERR_CUDA: return "CUDA error";
    case FE_ERR_OOM: return "out of memory";
    case FE_ERR_UNSUPPORTED: return "unsupported";
    case FE_ERR_NAN: return "NaN or Inf";
    case FE_ERR_NOT_CONVERGED: return "not converged";
    case FE_ERR_BREAKDOWN: return "breakdown";
    case FE_ERR_STATE: return "call out of order";
    }
    return "unknown";
}

extern "C" fe_status fe_num_dofs(const fe_ctx *c, int64_t *n_l, int64_t *n_free)
{
    if (!c) return FE_ERR_ARG;
    if (n_l) *n_l = c->nl;
    if (n_free) *n_free = c->nfree;
    return FE_OK;
}

extern "C" fe_status fe_num_elements(const fe_ctx *c, int64_t *n_e)
{
    if (!c || !n_e) return FE_ERR_ARG;
    *n_e = c->ne;
    return FE_OK;
}

extern "C" fe_status fe_memory_bytes(const fe_ctx *c, int64_t *bytes)
{
    if (!c || !bytes) return FE_ERR_ARG;
    *bytes = c->mem_bytes;
    return FE_OK;
}

// ------------------------------------------------------------------------------------------------
// operators
// ------------------------------------------------------------------------------------------------
extern "C" fe_status fe_residual(fe_ctx *c, const double *u, double *r, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!u || !r || u == r) return fail(c, FE_ERR_ARG, "fe_residual: null or aliased vectors");
    c->ops->residual(c, u, r, nullptr, nullptr, as_stream(stream));
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_linearize(fe_ctx *c, const double *u, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!u) return fail(c, FE_ERR_ARG, "fe_linearize: null u");
    fe_status s = ensure_tangent(c, true, true);
    if (s != FE_OK) return s;
    cudaStream_t st = as_stream(stream);
    c->ops->residual(c, u, nullptr, c->d_T64, c->d_T32, st);
    CKLAUNCH();
    c->ops->diag_64(c, c->d_diag, st);
    CKLAUNCH();
    c->lin64 = c->lin32 = c->have_diag = true;
    c->lindf = false;
    return FE_OK;
}

extern "C" fe_status fe_jacobian_action(fe_ctx *c, const double *u, const void *v, void *y, int precision,
                                        void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!v || !y || v == y) return fail(c, FE_ERR_ARG, "fe_jacobian_action: null or aliased vectors");
    cudaStream_t st = as_stream(stream);
    if (!u) return apply_jv_cached(c, v, y, precision, st);
    if (precision == 64) c->ops->jv_dual_64(c, u, (const double *)v, (double *)y, st);
    else if (precision == 32) c->ops->jv_dual_32(c, u, (const float *)v, (float *)y, st);
    else if (precision == -32) c->ops->jv_dual_32d(c, u, (const double *)v, (double *)y, st);
    else if (precision == 48)
        return fail(c, FE_ERR_UNSUPPORTED, "precision 48 applies to the cached linearisation only (u = NULL)");
    else return fail(c, FE_ERR_ARG, "precision must be 64, 48, 32 or -32");
    CKLAUNCH();
    return FE_OK;
}

namespace {

// The cached J v of a host vector in z-chunks of tile layers, so that the copies overlap the
// kernels: chunk c's DOF planes go to the device on one stream, its tiles run on `st` once they
// have landed, the fix-up rows of the planes that are then complete follow, and those planes go
// back on a third stream.  A tile layer L reads the DOF planes k T L .. k T (L + 1); after the
// layers below k T L1 have run (and the fix-up of their rows), the planes below k T L1 are final:
// the plane k T L1 itself still waits for its owner, the first layer of the next chunk.  The
// arithmetic is that of the one-piece action (the same kernels on the same tiles, the same
// fix-up rows in the same order), so the result is the same bit for bit.
fe_status jv_host_chunked(fe_ctx *c, const void *v_host, void *y_host, int precision, void *dv, void *dy,
                          cudaStream_t st)
{
    const size_t es = precision == 32 ? sizeof(float) : sizeof(double);
    const int64_t k = c->k, T = c->T;
    const int64_t mxy = ((int64_t)k * c->n[0] + 1) * ((int64_t)k * c->n[1] + 1);
    const int64_t zmax = (int64_t)k * c->n[2];                // last DOF plane
    const int64_t ntz = c->nt[2], ntxy = (int64_t)c->nt[0] * c->nt[1];
    // chunks: more of them shorten the pipeline's fill (the first chunk's copy in) and drain (the
    // last chunk's fix-up and copy back) but each costs launch tails and fix-up launches; at 64^3
    // order 3 (32 tile layers) 8 / 16 / 32 chunks took 1.971 / 1.939 / 1.926 ms per FP64 call, and
    // 0.63 / 0.77 / 1.17 ms per double-float and 0.58 / 0.61 / 0.87 ms per FP32-operator call,
    // whose actions are 4 and 12 times shorter
    const int nch = (int)std::min<int64_t>(precision == 64 ? 32 : 8, ntz);
    if (!c->cp_in) {
        CK(cudaStreamCreateWithFlags(&c->cp_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&c->cp_out, cudaStreamNonBlocking));
        // a chunk's fix-up takes the SM slots that free up before the next chunk's pending tiles
        // do, so that its rows go back to the host while that chunk computes
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        for (auto &t : c->cp_tile) CK(cudaStreamCreateWithPriority(&t, cudaStreamNonBlocking, lo));
        CK(cudaStreamCreateWithPriority(&c->cp_fix, cudaStreamNonBlocking, hi));
        for (auto &e : c->chunk_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &e : c->tile_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // the rows of each length class (1, 3, 7 halo entries), sorted by DOF within the class
    const int64_t cls0[3] = { 0, c->fix.n1, c->fix.n1 + c->fix.n3 };
    const int64_t cls1[3] = { c->fix.n1, c->fix.n1 + c->fix.n3, c->nfix };
    auto row_of = [&](int cl, int64_t g) {      // first row of class cl whose DOF is >= g
        const uint32_t *b = c->h_fix_g.data() + cls0[cl], *e = c->h_fix_g.data() + cls1[cl];
        return cls0[cl] + (int64_t)(std::lower_bound(b, e, (uint32_t)std::min<int64_t>(g, 0xFFFFFFFFll)) - b);
    };
    // the caller's stream work before this call, then the chunks
    CK(cudaEventRecord(c->chunk_ev[0], st));
    CK(cudaStreamWaitEvent(c->cp_in, c->chunk_ev[0], 0));
    int64_t in_end = 0, fin_end = 0;      // planes [0, in_end) sent, [0, fin_end) final
    for (int ch = 0; ch < nch; ++ch) {
        const int64_t L0 = ntz * ch / nch, L1 = ntz * (ch + 1) / nch;
        const bool last = ch == nch - 1;
        const int64_t need = last ? zmax + 1 : std::min(k * T * L1, zmax) + 1;
        const int64_t fin = last ? zmax + 1 : k * T * L1;
        cudaEvent_t ein = c->chunk_ev[1 + 2 * (ch % 8)], efin = c->chunk_ev[2 + 2 * (ch % 8)];
        if (need > in_end) {
            CK(cudaMemcpyAsync((char *)dv + in_end * mxy * es, (const char *)v_host + in_end * mxy * es,
                               (size_t)((need - in_end) * mxy) * es, cudaMemcpyHostToDevice, c->cp_in));
            in_end = need;
        }
        CK(cudaEventRecord(ein, c->cp_in));
        // the chunks' tile kernels alternate between two streams, so that one chunk's last wave
        // of tiles runs beside the next chunk's first: they write disjoint owned rows and halo
        // entries.  The fix-up of chunk ch (on cp_fix) waits for its tiles; the rows it completes
        // also hold the partial sums of chunk ch - 1's tiles, which cp_fix waited for before.
        cudaStream_t ts = c->cp_tile[ch % 2];
        CK(cudaStreamWaitEvent(ts, ein, 0));
        c->ops->jv_tiles(c, precision, dv, dy, L0 * ntxy, (L1 - L0) * ntxy, ts);
        CKLAUNCH();
        CK(cudaEventRecord(c->tile_ev[ch % 8], ts));
        CK(cudaStreamWaitEvent(c->cp_fix, c->tile_ev[ch % 8], 0));
        for (int cl = 0; cl < 3; ++cl) {
            const int64_t r0 = row_of(cl, fin_end * mxy), r1 = row_of(cl, fin * mxy);
            c->ops->fix_rows(c, precision, dy, r0, r1, c->cp_fix);
        }
        CKLAUNCH();
        CK(cudaEventRecord(efin, c->cp_fix));
        CK(cudaStreamWaitEvent(c->cp_out, efin, 0));
        if (fin > fin_end) {
            CK(cudaMemcpyAsync((char *)y_host + fin_end * mxy * es, (const char *)dy + fin_end * mxy * es,
                               (size_t)((fin - fin_end) * mxy) * es, cudaMemcpyDeviceToHost, c->cp_out));
            fin_end = fin;
        }
    }
    // the copies back belong to the call: `st` waits for them
    CK(cudaEventRecord(c->chunk_ev[0], c->cp_out));
    CK(cudaStreamWaitEvent(st, c->chunk_ev[0], 0));
    return FE_OK;
}

}  // namespace

extern "C" fe_status fe_jacobian_action_host(fe_ctx *c, const void *v_host, void *y_host, int precision,
                                             void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!v_host || !y_host) return fail(c, FE_ERR_ARG, "fe_jacobian_action_host: null buffers");
    const size_t es = precision == 32 ? sizeof(float) : sizeof(double);
    fe_status s = ensure_work(c);
    if (s != FE_OK) return s;
    cudaStream_t st = as_stream(stream);
    // the tile kernels of 3D problems with several tile layers: chunks that overlap the copies
    const int var = precision == 64 ? 0 : precision == 32 ? 1 : precision == -32 ? 2 : precision == 48 ? 3 : -1;
    if (var >= 0 && c->dim == 3 && c->pipe_grid[var] > 0 && c->nt[2] >= 2 && c->chunked_host) {
        if ((precision == 64 || precision == 48) && !c->lin64)
            return fail(c, FE_ERR_STATE, "no FP64 linearisation cached (call fe_linearize)");
        if ((precision == 32 || precision == -32) && !c->lin32)
            return fail(c, FE_ERR_STATE, "no FP32 linearisation cached (call fe_linearize)");
        if (precision == 48 && (s = prepare_tangent_df(c, st)) != FE_OK) return s;
        s = jv_host_chunked(c, v_host, y_host, precision, c->w_trial, c->w_d, st);
        if (s != FE_OK) return s;
        return check_device_error(c, st);
    }
    // staging in the CG work vectors (each holds N_L doubles)
    void *dv = c->w_trial, *dy = c->w_d;
    CK(cudaMemcpyAsync(dv, v_host, es * (size_t)c->nl, cudaMemcpyHostToDevice, st));
    s = apply_jv_cached(c, dv, dy, precision, st);
    if (s != FE_OK) return s;
    CK(cudaMemcpyAsync(y_host, dy, es * (size_t)c->nl, cudaMemcpyDeviceToHost, st));
    return check_device_error(c, st);
}

extern "C" fe_status fe_check_error(fe_ctx *c, void *stream)
{
    if (!c) return FE_ERR_ARG;
    return check_device_error(c, as_stream(stream));
}

extern "C" fe_status fe_selftest_wait_timeout(fe_ctx *c, void *stream)
{
    if (!c) return FE_ERR_ARG;
    cudaStream_t st = as_stream(stream);
    {
        LaunchScope ls(c, "wait_selftest", st);
        k_wait_selftest<<<1, 32, 0, st>>>(c->d_err);
    }
    CKLAUNCH();
    return check_device_error(c, st);
}

extern "C" fe_status fe_jacobian_diagonal(fe_ctx *c, double *diag, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!diag) return fail(c, FE_ERR_ARG, "fe_jacobian_diagonal: null output");
    if (!c->have_diag) return fail(c, FE_ERR_STATE, "no linearisation cached (call fe_linearize)");
    CK(cudaMemcpyAsync(diag, c->d_diag, (size_t)c->nl * sizeof(double), cudaMemcpyDeviceToDevice, as_stream(stream)));
    return FE_OK;
}

extern "C" fe_status fe_load_vector(fe_ctx *c, double *F, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!F) return fail(c, FE_ERR_ARG, "fe_load_vector: null output");
    fe_status s = ensure_work(c);
    if (s != FE_OK) return s;
    cudaStream_t st = as_stream(stream);
    // the flux vanishes at zero gradient, so R(0) = -F (essential entries 0)
    CK(cudaMemsetAsync(c->w_trial, 0, (size_t)c->nl * sizeof(double), st));
    c->ops->residual(c, c->w_trial, F, nullptr, nullptr, st);
    CKLAUNCH();
    {
        LaunchScope ls(c, "scale", st);
        k_scale<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(F, F, -1.0, c->nl);
    }
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_node_coords(fe_ctx *c, double *xyz, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!xyz) return fail(c, FE_ERR_ARG, "fe_node_coords: null output");
    cudaStream_t st = as_stream(stream);
    {
        LaunchScope ls(c, "node_coords", st);
        k_node_coords<<<(unsigned)((c->nl + 255) / 256), 256, 0, st>>>(c->gp, c->k, c->d_vert, xyz, c->nl);
    }
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_set_design(fe_ctx *c, const double *rho, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!rho) return fail(c, FE_ERR_ARG, "fe_set_design: null rho");
    if (!c->has_rho) return fail(c, FE_ERR_STATE, "context was set up without a design field");
    cudaStream_t st = as_stream(stream);
    CK(cudaMemcpyAsync(c->d_rho, rho, (size_t)c->ne * sizeof(double), cudaMemcpyDeviceToDevice, st));
    {
        LaunchScope ls(c, "design_factors", st);
        k_design_factors<<<(unsigned)((c->nepad + 255) / 256), 256, 0, st>>>(c->gp, c->d_rho, c->kappa_eps,
                                                                            c->kappa_q, c->d_kr, c->d_dkr);
    }
    CKLAUNCH();
    c->lin64 = c->lin32 = c->have_diag = c->lindf = false;
    return FE_OK;
}

extern "C" fe_status fe_adjoint_vjp(fe_ctx *c, const double *u, const double *lambda, double *grad_rho, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!u || !lambda || !grad_rho) return fail(c, FE_ERR_ARG, "fe_adjoint_vjp: null vectors");
    if (!c->has_rho) return fail(c, FE_ERR_STATE, "fe_adjoint_vjp needs a design field");
    c->ops->vjp(c, u, lambda, grad_rho, as_stream(stream));
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_compliance(fe_ctx *c, const double *u, double *out, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!u || !out) return fail(c, FE_ERR_ARG, "fe_compliance: null vectors");
    fe_status s = ensure_work(c);
    if (s != FE_OK) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = fe_load_vector(c, c->w_r, stream)) != FE_OK) return s;
    CgState *ds = cg_state(c) + 1;
    {
        LaunchScope ls(c, "dot", st);
        k_dot<<<RED_BLOCKS, RED_THREADS, 0, st>>>(c->w_r, u, c->nl, c->w_partial + 2 * RED_BLOCKS, &ds->counter, out);
    }
    CKLAUNCH();
    return FE_OK;
}

// ------------------------------------------------------------------------------------------------
// solvers
// ------------------------------------------------------------------------------------------------
extern "C" fe_status fe_cg_solve(fe_ctx *c, const double *b, double *x, double rtol, int max_iter, int precision,
                                 int *iters, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!b || !x || b == x) return fail(c, FE_ERR_ARG, "fe_cg_solve: null or aliased vectors");
    if (precision != 64 && precision != 48 && precision != 32 && precision != -32)
        return fail(c, FE_ERR_ARG, "precision must be 64, 48, 32 or -32");
    const bool f64 = precision == 64 || precision == 48;
    if ((f64 && !c->lin64) || (!f64 && !c->lin32) || !c->have_diag)
        return fail(c, FE_ERR_STATE, "no linearisation cached (call fe_linearize)");
    fe_status s = ensure_work(c);
    if (s != FE_OK) return s;
    CK(cudaStreamSynchronize(as_stream(stream)));
    cudaStream_t st = c->own_stream;
    if (precision == 48 && (s = prepare_tangent_df(c, st)) != FE_OK) return s;
    {
        LaunchScope ls(c, "reciprocal", st);
        k_reciprocal<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_dinv, c->w_dinv64, c->d_diag, c->nl);
    }
    CKLAUNCH();
    int it = 0, done = 0;
    s = run_cg(c, b, rtol, max_iter, precision, 16, 1, &it, &done);
    if (s != FE_OK) return s;
    CK(cudaMemcpyAsync(x, c->w_cx, (size_t)c->nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (iters) *iters = it;
    if (done == CG_BREAKDOWN) return fail(c, FE_ERR_BREAKDOWN, "CG breakdown (p^T J p <= 0)");
    if (done == CG_NAN) return fail(c, FE_ERR_NAN, "CG produced NaN/Inf");
    if (done == CG_MAXIT) return fail(c, FE_ERR_NOT_CONVERGED, "CG reached %d iterations", max_iter);
    return FE_OK;
}

extern "C" fe_status fe_compliance_gradient(fe_ctx *c, const double *u, double scale, double rtol, int max_iter,
                                            int precision, double *grad_rho, int *iters, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!u || !grad_rho) return fail(c, FE_ERR_ARG, "fe_compliance_gradient: null vectors");
    if (!c->has_rho) return fail(c, FE_ERR_STATE, "fe_compliance_gradient needs a design field");
    fe_status s = ensure_work(c);
    if (s != FE_OK) return s;
    cudaStream_t st = as_stream(stream);
    // J(u) lambda = F: the load vector in w_r, lambda in w_d (fe_cg_solve works in its own vectors)
    if ((s = fe_linearize(c, u, stream)) != FE_OK) return s;
    if ((s = fe_load_vector(c, c->w_r, stream)) != FE_OK) return s;
    if ((s = fe_cg_solve(c, c->w_r, c->w_d, rtol, max_iter, precision, iters, stream)) != FE_OK) return s;
    // fe_cg_solve ran on the context's own stream and synchronised it; the rest on `stream`
    c->ops->vjp(c, u, c->w_d, grad_rho, st);
    CKLAUNCH();
    {
        LaunchScope ls(c, "scale", st);
        k_scale<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(grad_rho, grad_rho, -scale, c->ne);
    }
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_newton_default_opts(fe_newton_opts *o)
{
    if (!o) return FE_ERR_ARG;
    o->rtol = 1e-8;
    o->max_newton = 50;
    o->max_cg = 20000;
    o->cg_rtol = 1e-4;
    o->inner_precision = 64;
    o->line_search = 1;
    o->armijo = 1e-4;
    o->max_halvings = 20;
    o->cg_batch = 16;
    o->use_graph = 2;
    o->forcing = 0;
    o->eta_max = 0.1;
    return FE_OK;
}

extern "C" fe_status newton_solve(fe_ctx *c, double *u, const fe_newton_opts *opts_in, fe_newton_report *rep,
                                  void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!u) return fail(c, FE_ERR_ARG, "newton_solve: null u");
    fe_newton_opts o;
    if (opts_in) o = *opts_in; else fe_newton_default_opts(&o);
    if (o.inner_precision != 64 && o.inner_precision != 48 && o.inner_precision != 32 && o.inner_precision != -32)
        return fail(c, FE_ERR_ARG, "inner_precision must be 64, 48, 32 or -32");
    if (o.forcing != 0 && o.forcing != 1) return fail(c, FE_ERR_ARG, "forcing must be 0 or 1");
    if (o.forcing == 1 && !(o.eta_max > 0.0 && o.eta_max < 1.0)) return fail(c, FE_ERR_ARG, "eta_max must lie in (0, 1)");
    fe_newton_report R;
    std::memset(&R, 0, sizeof R);
    // FP32 tangent for the FP32 operators; the FP64 one (split into FP32 word pairs before each CG
    // in mode 48) otherwise
    const bool mixed = o.inner_precision == 32 || o.inner_precision == -32;
    fe_status s = ensure_work(c);
    if (s == FE_OK) s = ensure_tangent(c, !mixed, mixed);
    if (s != FE_OK) return s;
    CK(cudaStreamSynchronize(as_stream(stream)));
    cudaStream_t st = c->own_stream;
    const int64_t l0 = c->launches;
    const auto t0 = std::chrono::steady_clock::now();
    double cg_ms = 0.0;
    double *T64 = mixed ? nullptr : c->d_T64;
    float *T32 = mixed ? c->d_T32 : nullptr;
    const int jprec = o.inner_precision;

    // R and J_D at u (fused)
    c->ops->residual(c, u, c->w_r, T64, T32, st);
    CKLAUNCH();
    double rr = 0.0;
    s = dot_sync(c, c->w_r, c->w_r, &rr, st);
    if (s != FE_OK) return s;
    double rnorm = std::sqrt(rr);
    R.r0 = rnorm;
    fe_status result = FE_OK;
    if (!std::isfinite(rnorm)) result = fail(c, FE_ERR_NAN, "initial residual is not finite");
    int it = 0;
    double rprev = rnorm, eta = o.cg_rtol;
    while (result == FE_OK && rnorm > o.rtol * R.r0 && R.r0 > 0.0) {
        if (it >= o.max_newton) { result = fail(c, FE_ERR_NOT_CONVERGED, "Newton reached %d steps", it); break; }
        // Jacobi preconditioner of the current linearisation
        if (mixed) c->ops->diag_32(c, c->d_diag, st); else c->ops->diag_64(c, c->d_diag, st);
        CKLAUNCH();
        {
            LaunchScope ls(c, "reciprocal", st);
            k_reciprocal<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_dinv, c->w_dinv64, c->d_diag, c->nl);
        }
        // right-hand side -R
        {
            LaunchScope ls(c, "scale", st);
            k_scale<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_d, c->w_r, -1.0, c->nl);
        }
        CKLAUNCH();
        if (jprec == 48) {
            c->lin64 = true;
            c->lindf = false;
            s = prepare_tangent_df(c, st);
            if (s != FE_OK) return s;
        }
        // inner tolerance: fixed, or the Eisenstat-Walker choice 2 forcing term
        if (o.forcing == 1) {
            if (it == 0) {
                eta = o.eta_max;
            } else {
                const double q = rnorm / rprev, keep = 0.9 * eta * eta;
                double e = 0.9 * q * q;
                if (keep > 0.1) e = std::max(e, keep);
                e = std::max(e, 0.5 * o.rtol * R.r0 / rnorm);
                eta = std::min(std::max(e, 1e-6), o.eta_max);
            }
        }
        const auto c0 = std::chrono::steady_clock::now();
        int cg_it = 0, done = 0;
        s = run_cg(c, c->w_d, eta, o.max_cg, jprec, o.cg_batch, o.use_graph, &cg_it, &done);
        if (s != FE_OK) return s;
        cg_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c0).count();
        R.cg_iters_total += cg_it;
        if (it < FE_NEWTON_HIST) R.cg_hist[it] = cg_it;
        if (done == CG_BREAKDOWN || done == CG_NAN) {
            result = fail(c, done == CG_NAN ? FE_ERR_NAN : FE_ERR_BREAKDOWN, "inner CG failed (%d)", done);
            break;
        }
        // backtracking line search on ||R||: trial = u + alpha d (d = CG solution in w_cx)
        double alpha = 1.0, tn = 0.0;
        bool accepted = false;
        for (int h = 0; h <= o.max_halvings; ++h) {
            {
                LaunchScope ls(c, "waxpy", st);
                k_waxpy<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(c->w_trial, u, alpha, c->w_cx, c->nl);
            }
            c->ops->residual(c, c->w_trial, c->w_d, T64, T32, st);
            CKLAUNCH();
            s = dot_sync(c, c->w_d, c->w_d, &tn, st);
            if (s != FE_OK) return s;
            tn = std::sqrt(tn);
            if (std::isfinite(tn) && (!o.line_search || tn <= (1.0 - o.armijo * alpha) * rnorm)) { accepted = true; break; }
            if (!o.line_search) break;
            alpha *= 0.5;
            R.line_search_halvings++;
        }
        if (!accepted) { result = fail(c, FE_ERR_BREAKDOWN, "line search failed at Newton step %d", it); break; }
        CK(cudaMemcpyAsync(u, c->w_trial, (size_t)c->nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::swap(c->w_r, c->w_d);
        rprev = rnorm;
        rnorm = tn;
        if (it < FE_NEWTON_HIST) R.r_hist[it] = rnorm;
        ++it;
    }
    CK(cudaStreamSynchronize(st));
    c->lin64 = !mixed; c->lin32 = mixed; c->have_diag = false; c->lindf = false;
    R.newton_iters = it;
    R.r_final = rnorm;
    R.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    R.t_cg_ms = cg_ms;
    R.kernel_launches = c->launches - l0;
    R.status = result;
    if (rep) *rep = R;
    return result;
}

// ------------------------------------------------------------------------------------------------
// profiling
// ------------------------------------------------------------------------------------------------
extern "C" fe_status fe_prof_enable(fe_ctx *c, int enable)
{
    if (!c) return FE_ERR_ARG;
    c->prof = enable != 0;
    return FE_OK;
}

extern "C" fe_status fe_prof_reset(fe_ctx *c)
{
    if (!c) return FE_ERR_ARG;
    CK(cudaDeviceSynchronize());
    for (auto &r : c->prof_recs) { c->prof_pool.push_back(r.a); c->prof_pool.push_back(r.b); }
    c->prof_recs.clear();
    std::fill(c->prof_count.begin(), c->prof_count.end(), 0);
    std::fill(c->prof_ms.begin(), c->prof_ms.end(), 0.0);
    c->launches = 0;
    return FE_OK;
}

extern "C" fe_status fe_prof_read(fe_ctx *c, int i, const char **name, int64_t *launches, double *ms, int *count)
{
    if (!c) return FE_ERR_ARG;
    if (!c->prof_recs.empty()) {
        CK(cudaDeviceSynchronize());
        for (auto &r : c->prof_recs) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, r.a, r.b));
            c->prof_ms[r.name] += t;
            c->prof_count[r.name] += 1;
            c->prof_pool.push_back(r.a);
            c->prof_pool.push_back(r.b);
        }
        c->prof_recs.clear();
    }
    if (count) *count = (int)c->prof_names.size();
    if (i >= 0 && i < (int)c->prof_names.size()) {
        if (name) *name = c->prof_names[i].c_str();
        if (launches) *launches = c->prof_count[i];
        if (ms) *ms = c->prof_ms[i];
    }
    return FE_OK;
}

extern "C" fe_status fe_launch_count(const fe_ctx *c, int64_t *launches)
{
    if (!c || !launches) return FE_ERR_ARG;
    *launches = c->launches;
    return FE_OK;
}

// ------------------------------------------------------------------------------------------------
// vector operations (the CG's building blocks, for solvers outside the library)
// ------------------------------------------------------------------------------------------------
extern "C" fe_status fe_dot(fe_ctx *c, const double *a, const double *b, int64_t begin, int64_t end, double *out,
                            void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!a || !b || !out || begin < 0 || end > c->nl || begin > end)
        return fail(c, FE_ERR_ARG, "fe_dot: null vectors or range outside [0, N_L]");
    fe_status s = ensure_work(c);
    if (s != FE_OK) return s;
    cudaStream_t st = as_stream(stream);
    CgState *ds = cg_state(c) + 1;
    {
        LaunchScope ls(c, "dot", st);
        k_dot<<<RED_BLOCKS, RED_THREADS, 0, st>>>(a + begin, b + begin, end - begin, c->w_partial + 2 * RED_BLOCKS,
                                                  &ds->counter, out);
    }
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_axpby(fe_ctx *c, double alpha, const double *x, double beta, double *y, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!x || !y) return fail(c, FE_ERR_ARG, "fe_axpby: null vectors");
    cudaStream_t st = as_stream(stream);
    {
        LaunchScope ls(c, "axpby", st);
        k_axpby<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(alpha, x, beta, y, c->nl);
    }
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_pointwise_mul(fe_ctx *c, const double *d, const double *r, double *z, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!d || !r || !z) return fail(c, FE_ERR_ARG, "fe_pointwise_mul: null vectors");
    cudaStream_t st = as_stream(stream);
    {
        LaunchScope ls(c, "pointwise_mul", st);
        k_mul<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(d, r, z, c->nl);
    }
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_reciprocal(fe_ctx *c, const double *x, double *y, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!x || !y) return fail(c, FE_ERR_ARG, "fe_reciprocal: null vectors");
    cudaStream_t st = as_stream(stream);
    {
        LaunchScope ls(c, "reciprocal", st);
        k_recip<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(x, y, c->nl);
    }
    CKLAUNCH();
    return FE_OK;
}

extern "C" fe_status fe_face_size(const fe_ctx *c, int face, int64_t *size)
{
    if (!c || !size || face < 0 || face >= 2 * c->dim) return FE_ERR_ARG;
    int64_t m[3] = { 1, 1, 1 };
    for (int d = 0; d < c->dim; ++d) m[d] = (int64_t)c->k * c->n[d] + 1;
    const int ax = face / 2;
    *size = m[0] * m[1] * m[2] / m[ax];
    return FE_OK;
}

extern "C" fe_status fe_face_add(fe_ctx *c, int face, double *y, const double *buf, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!y || !buf || face < 0 || face >= 2 * c->dim) return fail(c, FE_ERR_ARG, "fe_face_add: bad face or null vectors");
    FaceParams F{};
    F.dim = c->dim;
    F.face = face;
    F.natural = c->natural;
    for (int d = 0; d < 3; ++d) F.m[d] = d < c->dim ? (int64_t)c->k * c->n[d] + 1 : 1;
    int64_t size = 0;
    fe_face_size(c, face, &size);
    cudaStream_t st = as_stream(stream);
    {
        LaunchScope ls(c, "face_add", st);
        k_face_add<<<(unsigned)((size + 255) / 256), 256, 0, st>>>(F, y, buf);
    }
    CKLAUNCH();
    return FE_OK;
}

// ------------------------------------------------------------------------------------------------
// Jacobian action without allocation: scratch in a file-scope device array
// ------------------------------------------------------------------------------------------------
// Holds the cross-tile partial sums (the role of the context's halo buffer) for
// fe_jacobian_action_noalloc.  Every GPU that loads the library keeps it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FE_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

// Once per device, with that device current: the device address of the scratch array.  In host
// code the array's name is only a host-side stand-in, so kernels must be given this address.
fe_status noalloc_scratch_address(fe_ctx *c, int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(c, FE_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FE_OK;
}
}  // namespace

extern "C" fe_status fe_jacobian_action_noalloc(fe_ctx *c, const void *v, void *y, int precision, void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!v || !y || v == y) return fail(c, FE_ERR_ARG, "fe_jacobian_action_noalloc: null or aliased vectors");
    if (precision != 64 && precision != 32 && precision != -32)
        return fail(c, FE_ERR_ARG, "precision must be 64, 32 or -32");
    const size_t word = precision == 64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)c->nfixh * word;
    if (need > (size_t)FE_NOALLOC_SCRATCH_BYTES)
        return fail(c, FE_ERR_UNSUPPORTED,
                    "fe_jacobian_action_noalloc: problem needs %zu bytes of scratch, the static array holds %u",
                    need, (unsigned)FE_NOALLOC_SCRATCH_BYTES);
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(c, FE_ERR_ARG, "fe_jacobian_action_noalloc: current device %d is not the context's (%d)", dev,
                    c->device);
    if (dev < 0 || dev >= kMaxDevices)
        return fail(c, FE_ERR_ARG, "fe_jacobian_action_noalloc: device index %d beyond the %d the static-scratch "
                    "address table covers", dev, kMaxDevices);
    void *scratch = nullptr;
    fe_status s = noalloc_scratch_address(c, dev, &scratch);
    if (s != FE_OK) return s;
    // run the regular launchers with the static array standing in for the context's halo buffer
    void *own = c->d_halo;
    c->d_halo = scratch;
    s = apply_jv_cached(c, v, y, precision, as_stream(stream));
    c->d_halo = own;
    return s;
}
