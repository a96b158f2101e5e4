// batch.cu -- many independent instances (uneven size and order) in one persistent launch: the
// batched FP32 Jacobian action over a work list of (instance, tile) items, the batched fix-up,
// a segmented FP32 CG whose iterations replay as one captured CUDA graph for all instances, the
// lock-step FP64 Newton driver, and the autotuner that picks each order's tile edge and the
// persistent launch shape (cached in a JSON file).
#include <algorithm>
#include <cstdarg>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "element_kernels.cuh"
#include "vector_kernels.h"

namespace feod {

// ------------------------------------------------------------------------------------------------
// tile variants of the batched launch, two tile edges per order 1..4; every variant's thread count
// divides the CTA's 256 threads, so a CTA working on a variant splits into 256 / threads
// independent thread groups, one tile each
// ------------------------------------------------------------------------------------------------
constexpr int BATCH_MAX_ORDER = 4;
constexpr int NBV = 8;
constexpr int BATCH_THREADS = 256;
constexpr int MAX_SLOTS = 8;
constexpr int BV_D1[NBV] = { 2, 2, 3, 3, 4, 4, 5, 5 };
constexpr int BV_TT[NBV] = { 4, 2, 2, 1, 2, 1, 2, 1 };
__host__ __device__ constexpr int bv_threads(int v)
{
    return v == 0 ? TileShape<2, 4>::THREADS : v == 1 ? TileShape<2, 2>::THREADS
         : v == 2 ? TileShape<3, 2>::THREADS : v == 3 ? TileShape<3, 1>::THREADS
         : v == 4 ? TileShape<4, 2>::THREADS : v == 5 ? TileShape<4, 1>::THREADS
         : v == 6 ? TileShape<5, 2>::THREADS : TileShape<5, 1>::THREADS;
}
constexpr bool bv_all_divide()
{
    for (int v = 0; v < NBV; ++v)
        if (BATCH_THREADS % bv_threads(v) != 0 || BATCH_THREADS / bv_threads(v) > MAX_SLOTS) return false;
    return true;
}
static_assert(bv_all_divide(), "every batched variant must divide the CTA into at most MAX_SLOTS groups");
__host__ __device__ constexpr int bv_slots(int v) { return BATCH_THREADS / bv_threads(v); }
// bytes of one tile's shared region (without the mbarrier) for variant v
__host__ __device__ inline size_t bv_tile_bytes(int v, int64_t tqs)
{
    switch (v) {
    case 0: return tile2_smem_bytes<2, 4, float>(tqs) - 64;
    case 1: return tile2_smem_bytes<2, 2, float>(tqs) - 64;
    case 2: return tile2_smem_bytes<3, 2, float>(tqs) - 64;
    case 3: return tile2_smem_bytes<3, 1, float>(tqs) - 64;
    case 4: return tile2_smem_bytes<4, 2, float>(tqs) - 64;
    case 5: return tile2_smem_bytes<4, 1, float>(tqs) - 64;
    case 6: return tile2_smem_bytes<5, 2, float>(tqs) - 64;
    default: return tile2_smem_bytes<5, 1, float>(tqs) - 64;
    }
}
int bv_of(int order, int tile)
{
    for (int v = 0; v < NBV; ++v)
        if (BV_D1[v] == order + 1 && BV_TT[v] == tile) return v;
    return -1;
}
int bv_max_tile(int order)
{
    int t = -1;
    for (int v = 0; v < NBV; ++v)
        if (BV_D1[v] == order + 1 && BV_TT[v] > t) t = BV_TT[v];
    return t;
}
int bv_min_tile(int order)
{
    int t = 1 << 30;
    for (int v = 0; v < NBV; ++v)
        if (BV_D1[v] == order + 1 && BV_TT[v] < t) t = BV_TT[v];
    return t;
}
// the tile edge an instance of `order` with n elements per direction uses when `want` is asked
// for: want if it is compiled and fits (setup never takes a tile edge above n), else the largest
// compiled edge <= n; -1 if none fits
int fit_tile(int order, int want, int n)
{
    if (want <= n && bv_of(order, want) >= 0) return want;
    int best = -1;
    for (int v = 0; v < NBV; ++v)
        if (BV_D1[v] == order + 1 && BV_TT[v] <= n && BV_TT[v] > best) best = BV_TT[v];
    return best;
}

// Device descriptor of one instance.  v, y of the batched action are the batch vectors at off.
struct BatchInst {
    OpParams op;              // op.skip -> the instance's CG flag (or nullptr)
    const float *T32;
    float *halo;
    int64_t off;
    int variant;
    int order;
};

// The work list: every tile of every instance as an item (instance, tile), grouped by variant:
// items of variant v at [vbeg[v], vbeg[v+1]).  CTA b starts with variant start[b] and then takes
// the others in cyclic order.
struct Work {
    const int2 *items;
    int vbeg[NBV + 1];
    const unsigned char *start;
};

// FP32 basis pairs per order 1..4 (identical for every instance of an order, so one copy serves
// every batch).  In constant memory and indexed by each variant's compile-time order, the
// coefficients are operands of the multiply-adds, not loads.
__constant__ BasisPairs c_bpairs[BATCH_MAX_ORDER];

// One tile of a variant on one thread group, as a separate (not inlined) function: each variant
// keeps its own register allocation instead of the kernel taking the union of all of them.
template <int D1, int TT>
__device__ __noinline__ bool batch_item(const OpParams &P, const float *T32, const float *v, float *y, float *halo,
                                        int64_t t, unsigned char *sm, uint64_t *mbar, uint32_t parity, int tid,
                                        const GroupBar &bar)
{
    return tile2_body<D1, TT, float>(P, c_bpairs[D1 - 2], T32, v, y, halo, t, sm, mbar, parity, tid, bar);
}

// The persistent batched Jacobian action y = J v (FP32).  A CTA works on one variant at a time,
// split into 256 / threads independent thread groups; every group takes its next tile from the
// variant's counter (group leader's atomic, broadcast through shared memory under the group's
// named barrier 1 + g) and runs it with its own shared region and mbarrier g, whose phase bit is
// kept in shared memory.  Groups never wait for each other except when the CTA moves on to the
// next variant with work.  The batched fix-up resets the counters for the next launch.  Items of
// instances whose skip flag is set are passed over.
__global__ void __launch_bounds__(BATCH_THREADS, 4)
    k_jv_batch(const BatchInst *__restrict__ inst, const __grid_constant__ Work W, const float *__restrict__ vb,
               float *__restrict__ yb, int *err, unsigned *counters)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);       // MAX_SLOTS mbarriers in 64 bytes
    __shared__ uint32_t s_par[MAX_SLOTS];
    __shared__ int s_item[MAX_SLOTS];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < MAX_SLOTS; ++k) mbar_init(&mbar[k], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    if (tid < MAX_SLOTS) s_par[tid] = 0u;
    __syncthreads();
    const int v0 = W.start[blockIdx.x];
    for (int vi = 0; vi < NBV; ++vi) {
        const int v = (v0 + vi) % NBV;
        const int nv = W.vbeg[v + 1] - W.vbeg[v];
        if (nv == 0) continue;
        const int nthr = bv_threads(v);
        const int g = tid / nthr, lt = tid - g * nthr;
        const GroupBar bar{ 1 + g, nthr };
        uint64_t *mb = &mbar[g];
        for (;;) {
            if (lt == 0) s_item[g] = s_abort ? nv : (int)atomicAdd(&counters[v], 1u);
            bar.sync();
            const int idx = s_item[g];
            if (idx >= nv) break;
            const int2 it = W.items[W.vbeg[v] + idx];
            const BatchInst &I = inst[it.x];
            if (I.op.skip && *I.op.skip) {               // uniform in the group
                bar.sync();                              // all have read s_item[g] before the next write
                continue;
            }
            unsigned char *sm = smem + 64 + (size_t)g * bv_tile_bytes(v, I.op.tqs32);
            const float *vin = vb + I.off;
            float *y = yb + I.off;
            const uint32_t par = s_par[g];
            bool ok;
            switch (v) {
            case 0: ok = batch_item<2, 4>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            case 1: ok = batch_item<2, 2>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            case 2: ok = batch_item<3, 2>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            case 3: ok = batch_item<3, 1>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            case 4: ok = batch_item<4, 2>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            case 5: ok = batch_item<4, 1>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            case 6: ok = batch_item<5, 2>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            default: ok = batch_item<5, 1>(I.op, I.T32, vin, y, I.halo, it.y, sm, mb, par, lt, bar); break;
            }
            if (lt == 0) {
                if (ok) {
                    s_par[g] = par ^ 1u;                // this group's copy completed one phase
                } else {
                    // the tangent block did not land within the bound: report, let the copy finish,
                    // and stop taking items
                    atomicExch(err, 3);
                    mbar_wait_bounded(mb, par);
                    s_abort = 1;
                }
            }
            // this thread's shared-memory accesses are ordered before the group's next bulk copy,
            // which may land where this tile kept other arrays
            fence_proxy_async();
        }
        // every group is done with this variant before the CTA is re-partitioned for the next
        fence_proxy_async();
        __syncthreads();
        if (s_abort) break;
    }
}

// Work policy 3: one launch per tile variant.  CTA b runs item b of the variant's part of the work
// list with the variant's own thread count, shared memory and register allocation -- the shape of
// the single-instance tile kernel -- for the tiles of every instance of that variant.
template <int D1, int TT>
__global__ void __launch_bounds__(TileShape<D1, TT>::THREADS)
    k_jv_batch_variant(const BatchInst *__restrict__ inst, const int2 *__restrict__ items,
                       const float *__restrict__ vb, float *__restrict__ yb, int *err)
{
    const int2 it = items[blockIdx.x];
    const BatchInst &I = inst[it.x];
    if (I.op.skip && *I.op.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    // thread 0 initialises the barrier before it issues the copy; the other threads poll it only
    // after the body's first barrier
    if (!tile2_body<D1, TT, float>(I.op, c_bpairs[D1 - 2], I.T32, vb + I.off, yb + I.off, I.halo, it.y, smem + 64,
                                   mbar, 0u, tid, CtaBar{}) &&
        tid == 0) {
        // the tangent block did not land within the bound: report, let the copy finish
        atomicExch(err, 3);
        mbar_wait_bounded(mbar, 0);
    }
}

// the kernel of variant v (policy 3)
const void *bv_kernel(int v)
{
    switch (v) {
    case 0: return reinterpret_cast<const void *>(k_jv_batch_variant<2, 4>);
    case 1: return reinterpret_cast<const void *>(k_jv_batch_variant<2, 2>);
    case 2: return reinterpret_cast<const void *>(k_jv_batch_variant<3, 2>);
    case 3: return reinterpret_cast<const void *>(k_jv_batch_variant<3, 1>);
    case 4: return reinterpret_cast<const void *>(k_jv_batch_variant<4, 2>);
    case 5: return reinterpret_cast<const void *>(k_jv_batch_variant<4, 1>);
    case 6: return reinterpret_cast<const void *>(k_jv_batch_variant<5, 2>);
    default: return reinterpret_cast<const void *>(k_jv_batch_variant<5, 1>);
    }
}

// Batched fix-up: row r of the concatenated fix-up rows belongs to the instance i with
// row0[i] <= r < row0[i+1] (binary search over the instances).
struct BatchFix {
    FixParams fix;
    const float *halo;
    int64_t off;
};

// blk_inst: per block, the instance of its first row (the largest i with row0[i] <= that row); a
// row's instance is found from there by a forward scan over row0 (a block's rows span few
// instances) instead of a binary search over all of them
__global__ void k_fixup_batch(const BatchFix *__restrict__ bf, const int64_t *__restrict__ row0, int count,
                              const int *__restrict__ blk_inst, float *__restrict__ yb, unsigned *counter)
{
    // the batched action before this kernel has taken all its items: reset its counters
    if (blockIdx.x == 0 && threadIdx.x < NBV) counter[threadIdx.x] = 0u;
    const int64_t nrows = row0[count];
    const int64_t rb = (int64_t)blockIdx.x * FIX_ROWS * blockDim.x + threadIdx.x;
    // FIX_ROWS rows per thread, their loads issued before their use (as k_fixup)
    float *yp[FIX_ROWS];
    const float *hp[FIX_ROWS];
    uint32_t g[FIX_ROWS], j0[FIX_ROWS], j1[FIX_ROWS];
#pragma unroll
    for (int i = 0; i < FIX_ROWS; ++i) {
        const int64_t r = rb + (int64_t)i * blockDim.x;
        j0[i] = j1[i] = 0u; g[i] = 0u; yp[i] = yb; hp[i] = nullptr;
        if (r >= nrows) continue;
        int lo = blk_inst[blockIdx.x];   // the largest lo with row0[lo] <= r
        while (lo + 1 < count && row0[lo + 1] <= r) ++lo;
        const BatchFix &B = bf[lo];
        if (B.fix.skip && *B.fix.skip) continue;
        const int64_t rr = r - row0[lo];
        uint32_t first, cnt;
        fix_entries(B.fix, rr, first, cnt);
        g[i] = B.fix.fix_g[rr];
        j0[i] = first;
        j1[i] = first + cnt;
        yp[i] = yb + B.off;
        hp[i] = B.halo;
    }
    float acc[FIX_ROWS];
    uint32_t kmax = 0;
#pragma unroll
    for (int i = 0; i < FIX_ROWS; ++i) {
        acc[i] = j1[i] > j0[i] ? yp[i][g[i]] : 0.f;
        kmax = max(kmax, j1[i] - j0[i]);
    }
    for (uint32_t k = 0; k < kmax; ++k) {
        float h[FIX_ROWS];
#pragma unroll
        for (int i = 0; i < FIX_ROWS; ++i) h[i] = j0[i] + k < j1[i] ? hp[i][j0[i] + k] : 0.f;
#pragma unroll
        for (int i = 0; i < FIX_ROWS; ++i)
            if (j0[i] + k < j1[i]) acc[i] += h[i];
    }
#pragma unroll
    for (int i = 0; i < FIX_ROWS; ++i)
        if (j1[i] > j0[i]) yp[i][g[i]] = acc[i];
}

// ------------------------------------------------------------------------------------------------
// segmented vector kernels: block b works on elements [lo[b], hi[b]) of instance inst[b]; the
// per-instance sums go through partial[b] and the instance's last-block ticket, in a fixed order
// ------------------------------------------------------------------------------------------------
constexpr int SEG_THREADS = 256;
constexpr int SEG_CHUNK = 8192;

struct Seg {
    const int *inst;          // [nblk]
    const int64_t *lo, *hi;   // [nblk]
    const int *blk0;          // [count+1] first block of each instance
};

__device__ __forceinline__ double seg_block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = SEG_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Sums NSUM values over the blocks of instance i (fixed order); true in every thread of the
// instance's last block, with the sums in out (valid in all threads).
template <int NSUM>
__device__ __forceinline__ bool seg_last_sum(const Seg &S, int i, const double (&mine)[NSUM], double *partial,
                                             int nblk, unsigned *counter, double (&out)[NSUM], double *sh)
{
    __shared__ bool is_last;
    for (int k = 0; k < NSUM; ++k) {
        const double b = seg_block_sum(mine[k], sh);
        if (threadIdx.x == 0) partial[(int64_t)k * nblk + blockIdx.x] = b;
    }
    const int b0 = S.blk0[i], b1 = S.blk0[i + 1];
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = atomicAdd(counter, 1u) == (unsigned)(b1 - b0 - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    for (int k = 0; k < NSUM; ++k) {
        double v = 0.0;
        for (int b = b0 + threadIdx.x; b < b1; b += SEG_THREADS) v += ((volatile double *)partial)[(int64_t)k * nblk + b];
        out[k] = seg_block_sum(v, sh);
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// FP64 segmented dot: st[i].scalar = a_i . b_i
__global__ void __launch_bounds__(SEG_THREADS) k_bdot64(const double *__restrict__ a, const double *__restrict__ b,
                                                        const Seg S, int nblk, CgState *st, double *partial)
{
    __shared__ double sh[SEG_THREADS];
    const int i = S.inst[blockIdx.x];
    double s[1] = { 0.0 }, o[1];
    for (int64_t k = S.lo[blockIdx.x] + threadIdx.x; k < S.hi[blockIdx.x]; k += SEG_THREADS) s[0] += a[k] * b[k];
    if (seg_last_sum<1>(S, i, s, partial, nblk, &st[i].counter, o, sh) && threadIdx.x == 0) st[i].scalar = o[0];
}

struct Acc2b {
    float s = 0.0f, c = 0.0f;
};
// compensated FP32 dot product step (Ogita-Rump-Oishi Dot2: TwoProduct by FMA, TwoSum)
__device__ __forceinline__ void acc2b(Acc2b &a, float x, float y)
{
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    const float s = __fadd_rn(a.s, p);
    const float z = __fsub_rn(s, a.s);
    const float se = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, z)), __fsub_rn(p, z));
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(pe, se));
}
__device__ __forceinline__ double acc2b_value(const Acc2b &a) { return (double)a.s + (double)a.c; }

// CG start for every instance (x = 0): instances with active[i] == 0 are marked converged.
// b is scaled by 2^e_i near its RMS (bb from k_bdot64 in st[i].scalar).
__global__ void __launch_bounds__(SEG_THREADS) k_bcg_init32(const double *__restrict__ b, const float *__restrict__ dinv,
                                                            float *__restrict__ x, float *__restrict__ r,
                                                            float *__restrict__ p, const Seg S, int nblk,
                                                            const int64_t *__restrict__ len, const int *__restrict__ active,
                                                            CgState *st, double rtol, int max_iter, double *partial)
{
    __shared__ double sh[SEG_THREADS];
    const int i = S.inst[blockIdx.x];
    const double bb = st[i].scalar;
    int e = 0;
    if (bb > 0.0 && isfinite(bb)) frexp(sqrt(bb / (double)len[i]), &e);
    Acc2b rz, rr;
    for (int64_t k = S.lo[blockIdx.x] + threadIdx.x; k < S.hi[blockIdx.x]; k += SEG_THREADS) {
        const float ri = (float)ldexp(b[k], -e);
        const float zi = __fmul_rn(dinv[k], ri);
        x[k] = 0.0f; r[k] = ri; p[k] = zi;
        acc2b(rz, ri, zi); acc2b(rr, ri, ri);
    }
    double s[2] = { acc2b_value(rz), acc2b_value(rr) }, o[2];
    if (seg_last_sum<2>(S, i, s, partial, nblk, &st[i].counter, o, sh) && threadIdx.x == 0) {
        CgState &T = st[i];
        T.scale_exp = e;
        T.rz = o[0]; T.rr = o[1]; T.rr0 = o[1];
        T.tol2 = rtol * rtol * o[1];
        T.iter = 0; T.max_iter = max_iter;
        T.done = !active[i] ? CG_CONVERGED
               : (o[1] <= T.tol2 || o[1] == 0.0) ? CG_CONVERGED : (isfinite(o[1]) ? 0 : CG_NAN);
        if (max_iter <= 0 && !T.done) T.done = CG_MAXIT;
    }
}

__global__ void __launch_bounds__(SEG_THREADS) k_bcg_alpha32(const float *__restrict__ p, const float *__restrict__ q,
                                                             const Seg S, int nblk, CgState *st, double *partial)
{
    const int i = S.inst[blockIdx.x];
    if (st[i].done) return;
    __shared__ double sh[SEG_THREADS];
    Acc2b pq;
    for (int64_t k = S.lo[blockIdx.x] + threadIdx.x; k < S.hi[blockIdx.x]; k += SEG_THREADS) acc2b(pq, p[k], q[k]);
    double s[1] = { acc2b_value(pq) }, o[1];
    if (seg_last_sum<1>(S, i, s, partial, nblk, &st[i].counter, o, sh) && threadIdx.x == 0) {
        CgState &T = st[i];
        T.pq = o[0];
        if (!(o[0] > 0.0) || !isfinite(o[0])) { T.done = CG_BREAKDOWN; T.alpha = 0.0; }
        else T.alpha = T.rz / o[0];
    }
}

__global__ void __launch_bounds__(SEG_THREADS) k_bcg_update32(float *__restrict__ x, float *__restrict__ r,
                                                              const float *__restrict__ p, const float *__restrict__ q,
                                                              const float *__restrict__ dinv, const Seg S, int nblk,
                                                              CgState *st, double *partial)
{
    const int i = S.inst[blockIdx.x];
    if (st[i].done) return;
    __shared__ double sh[SEG_THREADS];
    const float alpha = (float)st[i].alpha;
    Acc2b rz, rr;
    for (int64_t k = S.lo[blockIdx.x] + threadIdx.x; k < S.hi[blockIdx.x]; k += SEG_THREADS) {
        x[k] = __fmaf_rn(alpha, p[k], x[k]);
        const float ri = __fmaf_rn(-alpha, q[k], r[k]);
        r[k] = ri;
        const float zi = __fmul_rn(dinv[k], ri);
        acc2b(rz, ri, zi); acc2b(rr, ri, ri);
    }
    double s[2] = { acc2b_value(rz), acc2b_value(rr) }, o[2];
    if (seg_last_sum<2>(S, i, s, partial, nblk, &st[i].counter, o, sh) && threadIdx.x == 0) {
        CgState &T = st[i];
        T.beta = o[0] / T.rz;
        T.rz = o[0]; T.rr = o[1];
        T.iter += 1;
        if (!isfinite(o[1])) T.done = CG_NAN;
        else if (o[1] <= T.tol2) T.done = CG_CONVERGED;
        else if (T.iter >= T.max_iter) T.done = CG_MAXIT;
    }
}

__global__ void __launch_bounds__(SEG_THREADS) k_bcg_direction32(float *__restrict__ p, const float *__restrict__ r,
                                                                 const float *__restrict__ dinv, const Seg S,
                                                                 const CgState *st)
{
    const int i = S.inst[blockIdx.x];
    if (st[i].done) return;
    const float beta = (float)st[i].beta;
    for (int64_t k = S.lo[blockIdx.x] + threadIdx.x; k < S.hi[blockIdx.x]; k += SEG_THREADS)
        p[k] = __fmaf_rn(beta, p[k], __fmul_rn(dinv[k], r[k]));
}

// The condition of the device-side batched CG loop (a conditional WHILE node): repeat the body
// while any instance's CG is running.  One warp; the body's kernels have finished when it runs.
__global__ void k_bcg_continue(cudaGraphConditionalHandle h, const CgState *st, int count)
{
    int running = 0;
    for (int i = threadIdx.x; i < count; i += 32) running |= st[i].done == 0;
    running = __any_sync(0xffffffffu, running);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, running ? 1u : 0u);
}

// d = 2^e_i x in FP64: instance i's FP32 CG solution of its scaled system, unscaled (exact)
__global__ void __launch_bounds__(SEG_THREADS) k_bcg_widen(double *__restrict__ d, const float *__restrict__ x,
                                                           const Seg S, const CgState *st)
{
    const int i = S.inst[blockIdx.x];
    const double sc = ldexp(1.0, st[i].scale_exp);
    for (int64_t k = S.lo[blockIdx.x] + threadIdx.x; k < S.hi[blockIdx.x]; k += SEG_THREADS) d[k] = (double)x[k] * sc;
}

// b = -R (the Newton right-hand sides) and the FP32 Jacobi scaling dinv = 1 / diag(J)
__global__ void k_neg_recip(double *__restrict__ b, const double *__restrict__ r, float *__restrict__ dinv,
                            const double *__restrict__ diag, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        b[k] = -r[k];
        const double dg = diag[k];
        dinv[k] = (float)(dg != 0.0 ? 1.0 / dg : 1.0);
    }
}

// out = u + a d (a line-search trial point)
__global__ void k_axpy_to(double *__restrict__ out, const double *__restrict__ u, double a,
                          const double *__restrict__ d, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = u[k] + a * d[k];
}

}  // namespace feod

using namespace feod;

// ------------------------------------------------------------------------------------------------
// host runtime
// ------------------------------------------------------------------------------------------------
struct fe_batch {
    int count = 0;
    int device = 0, num_sms = 0;
    std::vector<fe_ctx *> ctx;
    std::vector<int> order, tile, variant;
    std::vector<int64_t> off, len;        // instance segments of the batch vectors
    int64_t total = 0;
    // launch shape (autotuned)
    int grid = 0, threads = 0, policy = 0;
    size_t smem = 0;
    size_t vsmem[NBV] = {};               // policy 3: dynamic shared memory of each variant's launch
    int ntotal_items = 0;
    int vbeg[NBV + 1] = {};
    // device data
    BatchInst *d_inst = nullptr;          // two copies: [0, count) skip -> CG flags; [count, 2 count) none
    int2 *d_items = nullptr;              // work items grouped by variant
    unsigned char *d_start = nullptr;     // first variant of each CTA
    unsigned *d_counter = nullptr;        // per-variant item counters of the batched action
    BatchFix *d_fix = nullptr;            // same two copies
    int64_t *d_row0 = nullptr;
    int *d_fix_blk = nullptr;             // per fix-up block, the instance of its first row
    int64_t nrows = 0;
    int *d_seg_inst = nullptr, *d_blk0 = nullptr;
    int64_t *d_seg_lo = nullptr, *d_seg_hi = nullptr, *d_len = nullptr;
    int nblk = 0;
    int *d_active = nullptr, *d_err = nullptr;
    CgState *d_state = nullptr;
    CgState *h_state = nullptr;           // pinned
    double *d_partial = nullptr;
    float *fx = nullptr, *fr = nullptr, *fp = nullptr, *fq = nullptr, *dinv = nullptr;
    double *R = nullptr, *Rt = nullptr, *B = nullptr, *D = nullptr, *diag = nullptr;
    cudaStream_t st = nullptr;
    // policy 3: each variant's launch on a stream of its own between a fork and a join on the
    // caller's stream, so that the launches run side by side (they write disjoint rows and halo
    // entries) instead of each waiting for the previous one's last wave
    cudaStream_t vst[NBV] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[NBV] = {};
    cudaGraphExec_t cg_exec = nullptr;    // one CG batch (use_graph 1)
    int cg_batch = 0;
    cudaGraphExec_t cg_loop = nullptr;    // the whole CG on the device (use_graph 2)
    int cg_loop_m = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

fe_status bfail(fe_batch *b, fe_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
fe_status bfail(fe_batch *b, fe_status s, const char *fmt, ...)
{
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        b->err = buf;
    }
    return s;
}

#define BCK(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA, "%s: %s (%s:%d)",  \
                         #call, cudaGetErrorString(e_), __FILE__, __LINE__);                             \
    } while (0)

#define BCKS(call)                                                                                        \
    do {                                                                                                  \
        fe_status s_ = (call);                                                                            \
        if (s_ != FE_OK) return s_;                                                                       \
    } while (0)

template <typename T>
cudaError_t balloc(T **p, size_t n) { return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T)); }

std::string g_batch_setup_error;

// --- tiny JSON cache: {"key": {"ms": [..], "best": ..}, ...} as flat "key": value lines ---------------
// The cache maps "<gpu>|<what>" to a number; it is written as a flat JSON object.
struct TuneCache {
    std::vector<std::pair<std::string, double>> kv;
    bool load(const char *path)
    {
        kv.clear();
        FILE *f = path ? std::fopen(path, "r") : nullptr;
        if (!f) return false;
        std::string s;
        char buf[4096];
        size_t n;
        while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
        std::fclose(f);
        size_t i = 0;
        while ((i = s.find('"', i)) != std::string::npos) {
            const size_t j = s.find('"', i + 1);
            if (j == std::string::npos) break;
            const std::string key = s.substr(i + 1, j - i - 1);
            const size_t c = s.find(':', j);
            if (c == std::string::npos) break;
            char *end = nullptr;
            const double v = std::strtod(s.c_str() + c + 1, &end);
            if (end == s.c_str() + c + 1) break;
            kv.emplace_back(key, v);
            i = (size_t)(end - s.c_str());
        }
        return true;
    }
    bool get(const std::string &k, double *v) const
    {
        for (auto &e : kv)
            if (e.first == k) { *v = e.second; return true; }
        return false;
    }
    void set(const std::string &k, double v)
    {
        for (auto &e : kv)
            if (e.first == k) { e.second = v; return; }
        kv.emplace_back(k, v);
    }
    bool save(const char *path) const
    {
        if (!path) return false;
        FILE *f = std::fopen(path, "w");
        if (!f) return false;
        std::fprintf(f, "{\n");
        for (size_t i = 0; i < kv.size(); ++i)
            std::fprintf(f, "  \"%s\": %.17g%s\n", kv[i].first.c_str(), kv[i].second, i + 1 < kv.size() ? "," : "");
        std::fprintf(f, "}\n");
        std::fclose(f);
        return true;
    }
};

void free_batch_device(fe_batch *b)
{
    void *ptrs[] = { b->d_inst, b->d_items, b->d_start, b->d_counter, b->d_fix, b->d_row0, b->d_fix_blk, b->d_seg_inst, b->d_blk0, b->d_seg_lo, b->d_seg_hi,
                     b->d_len, b->d_active, b->d_err, b->d_state, b->d_partial, b->fx, b->fr, b->fp, b->fq, b->dinv,
                     b->R, b->Rt, b->B, b->D, b->diag };
    for (void *p : ptrs)
        if (p) cudaFree(p);
    b->d_inst = nullptr; b->d_items = nullptr; b->d_start = nullptr; b->d_counter = nullptr; b->d_fix = nullptr; b->d_row0 = nullptr; b->d_seg_inst = nullptr;
    b->d_fix_blk = nullptr;
    b->d_blk0 = nullptr; b->d_seg_lo = nullptr; b->d_seg_hi = nullptr; b->d_len = nullptr; b->d_active = nullptr;
    b->d_err = nullptr; b->d_state = nullptr; b->d_partial = nullptr; b->fx = b->fr = b->fp = b->fq = b->dinv = nullptr;
    b->R = b->Rt = b->B = b->D = b->diag = nullptr;
}

// the work list: every tile of every instance, grouped by variant; within a variant, by policy
//   0: instance by instance;  1: interleaved (each instance's tiles spread evenly over the list);
//   2: instances by decreasing DOF count (the largest first, the small ones fill the tail)
//   3: as 0, run as one launch per variant (k_jv_batch_variant) instead of the persistent kernel
// and the first variant of every CTA, in proportion to the variants' estimated work
fe_status upload_work(fe_batch *b, int policy)
{
    const int n = b->count;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    if (policy == 2)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->len[x] > b->len[y]; });
    std::vector<std::vector<int2>> per(NBV);
    for (int v = 0; v < NBV; ++v) {
        std::vector<int> mine;
        for (int i : order)
            if (b->variant[i] == v) mine.push_back(i);
        if (policy != 1) {
            for (int i : mine)
                for (int64_t t = 0; t < b->ctx[i]->ntiles; ++t) per[v].push_back(make_int2(i, (int)t));
        } else {
            std::vector<int64_t> next(mine.size(), 0);
            std::vector<double> pos(mine.size());
            int64_t tot = 0;
            for (size_t j = 0; j < mine.size(); ++j) {
                tot += b->ctx[mine[j]]->ntiles;
                pos[j] = 0.5 / (double)b->ctx[mine[j]]->ntiles;
            }
            for (int64_t k = 0; k < tot; ++k) {
                size_t best = 0;
                for (size_t j = 1; j < mine.size(); ++j)
                    if (pos[j] < pos[best]) best = j;
                const int i = mine[best];
                per[v].push_back(make_int2(i, (int)next[best]));
                next[best]++;
                pos[best] = next[best] < b->ctx[i]->ntiles ? (next[best] + 0.5) / (double)b->ctx[i]->ntiles : 2.0;
            }
        }
    }
    std::vector<int2> items;
    double work[NBV];
    for (int v = 0; v < NBV; ++v) {
        b->vbeg[v] = (int)items.size();
        items.insert(items.end(), per[v].begin(), per[v].end());
        // a tile's cost grows with its elements and the contraction length: T^3 D1^4
        work[v] = (double)per[v].size() * BV_TT[v] * BV_TT[v] * BV_TT[v] * std::pow((double)BV_D1[v], 4.0);
    }
    b->vbeg[NBV] = (int)items.size();
    b->ntotal_items = (int)items.size();
    if (b->d_items) { cudaFree(b->d_items); b->d_items = nullptr; }
    BCK(balloc(&b->d_items, items.size()));
    BCK(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
    // CTA b starts where the cumulative work share passes (b + 1/2) / grid
    double wt = 0.0;
    for (int v = 0; v < NBV; ++v) wt += work[v];
    std::vector<unsigned char> start(std::max(b->grid, 1), 0);
    for (int c = 0; c < b->grid; ++c) {
        const double f = (c + 0.5) / b->grid * wt;
        double acc = 0.0;
        int v = 0;
        for (; v < NBV - 1; ++v) {
            acc += work[v];
            if (f < acc && work[v] > 0) break;
        }
        while (work[v] == 0.0 && v > 0) --v;
        start[c] = (unsigned char)v;
    }
    if (b->d_start) { cudaFree(b->d_start); b->d_start = nullptr; }
    BCK(balloc(&b->d_start, start.size()));
    BCK(cudaMemcpy(b->d_start, start.data(), start.size(), cudaMemcpyHostToDevice));
    b->policy = policy;
    return FE_OK;
}

// batched action on the batch vectors vb -> yb; with_skip: items of converged instances skipped
fe_status launch_jv(fe_batch *b, const float *vb, float *yb, bool with_skip, cudaStream_t st)
{
    const BatchInst *inst = b->d_inst + (with_skip ? 0 : b->count);
    const BatchFix *fix = b->d_fix + (with_skip ? 0 : b->count);
    Work W;
    W.items = b->d_items;
    for (int v = 0; v <= NBV; ++v) W.vbeg[v] = b->vbeg[v];
    W.start = b->d_start;
    if (b->policy == 3) {
        BCK(cudaEventRecord(b->fork_ev, st));
        for (int v = 0; v < NBV; ++v) {
            const int nv = b->vbeg[v + 1] - b->vbeg[v];
            if (nv == 0) continue;
            const int2 *items = b->d_items + b->vbeg[v];
            void *args[] = { (void *)&inst, (void *)&items, (void *)&vb, (void *)&yb, (void *)&b->d_err };
            BCK(cudaStreamWaitEvent(b->vst[v], b->fork_ev, 0));
            BCK(cudaLaunchKernel(bv_kernel(v), dim3((unsigned)nv), dim3((unsigned)bv_threads(v)), args, b->vsmem[v],
                                 b->vst[v]));
            BCK(cudaEventRecord(b->join_ev[v], b->vst[v]));
            BCK(cudaStreamWaitEvent(st, b->join_ev[v], 0));
            b->launches += 1;
        }
    } else {
        k_jv_batch<<<b->grid, BATCH_THREADS, b->smem, st>>>(inst, W, vb, yb, b->d_err, b->d_counter);
        b->launches += 1;
    }
    const unsigned fb = (unsigned)std::max<int64_t>(1, (b->nrows + 256 * FIX_ROWS - 1) / (256 * FIX_ROWS));
    k_fixup_batch<<<fb, 256, 0, st>>>(fix, b->d_row0, b->count, b->d_fix_blk, yb, b->d_counter);
    b->launches += 1;
    BCK(cudaGetLastError());
    return FE_OK;
}

// time `reps` batched actions (CUDA events), milliseconds per action
fe_status time_jv(fe_batch *b, int reps, double *ms)
{
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    BCKS(launch_jv(b, b->fp, b->fq, false, b->st));
    BCK(cudaEventRecord(e0, b->st));
    for (int r = 0; r < reps; ++r) BCKS(launch_jv(b, b->fp, b->fq, false, b->st));
    BCK(cudaEventRecord(e1, b->st));
    BCK(cudaEventSynchronize(e1));
    float t = 0.f;
    BCK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / reps;
    return FE_OK;
}

// (re)build the per-instance descriptors, fix-up tables, segments and launch shape; contexts exist
fe_status build_tables(fe_batch *b)
{
    const int n = b->count;
    free_batch_device(b);
    b->off.assign(n + 1, 0);
    b->len.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        b->len[i] = b->ctx[i]->nl;
        b->off[i + 1] = b->off[i] + ((b->len[i] + 63) / 64) * 64;   // 256-byte aligned segments
    }
    b->total = b->off[n];
    BCK(balloc(&b->d_err, 1));
    BCK(cudaMemset(b->d_err, 0, sizeof(int)));
    BCK(balloc(&b->d_counter, NBV));
    BCK(cudaMemset(b->d_counter, 0, NBV * sizeof(unsigned)));
    BCK(balloc(&b->d_state, n));
    BCK(cudaMemset(b->d_state, 0, n * sizeof(CgState)));
    if (!b->h_state) BCK(cudaMallocHost(&b->h_state, n * sizeof(CgState)));
    // instance descriptors: copy [0, n) with the CG flags, [n, 2n) without
    std::vector<BatchInst> hi(2 * n);
    std::vector<BatchFix> hf(2 * n);
    std::vector<int64_t> row0(n + 1, 0);
    size_t smem = 64;
    int threads = 32;
    for (int i = 0; i < n; ++i) {
        fe_ctx *c = b->ctx[i];
        // the descriptors hold the tangent's address: allocate it (zero-filled) first
        BCKS(alloc_tangent32(c));
        if (!c->d_T32 || !c->d_halo) return bfail(b, FE_ERR_STATE, "instance %d has no tangent or halo storage", i);
        BatchInst I{};
        I.op = c->op;
        I.op.err = b->d_err;
        I.T32 = c->d_T32;
        I.halo = reinterpret_cast<float *>(c->d_halo);
        I.off = b->off[i];
        I.variant = b->variant[i];
        I.order = b->order[i];
        hi[n + i] = I;
        hi[n + i].op.skip = nullptr;
        I.op.skip = &b->d_state[i].done;
        hi[i] = I;
        BatchFix F{};
        F.fix = c->fix;
        F.halo = reinterpret_cast<const float *>(c->d_halo);
        F.off = b->off[i];
        hf[n + i] = F;
        hf[n + i].fix.skip = nullptr;
        F.fix.skip = &b->d_state[i].done;
        hf[i] = F;
        row0[i + 1] = row0[i] + c->nfix;
        smem = std::max(smem, 64 + (size_t)bv_slots(b->variant[i]) * bv_tile_bytes(b->variant[i], c->tqs32));
        threads = BATCH_THREADS;
    }
    b->nrows = row0[n];
    b->smem = smem;
    b->threads = threads;
    BCK(balloc(&b->d_inst, 2 * n));
    BCK(cudaMemcpy(b->d_inst, hi.data(), hi.size() * sizeof(BatchInst), cudaMemcpyHostToDevice));
    BCK(balloc(&b->d_fix, 2 * n));
    BCK(cudaMemcpy(b->d_fix, hf.data(), hf.size() * sizeof(BatchFix), cudaMemcpyHostToDevice));
    BCK(balloc(&b->d_row0, n + 1));
    BCK(cudaMemcpy(b->d_row0, row0.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    {
        // the fix-up's blocks take 256 FIX_ROWS consecutive rows each (launch_jv)
        const int64_t per = 256 * FIX_ROWS, nb = std::max<int64_t>(1, (b->nrows + per - 1) / per);
        std::vector<int> fb((size_t)nb);
        int lo = 0;
        for (int64_t j = 0; j < nb; ++j) {
            while (lo + 1 < n && row0[lo + 1] <= j * per) ++lo;
            fb[(size_t)j] = lo;
        }
        BCK(balloc(&b->d_fix_blk, nb));
        BCK(cudaMemcpy(b->d_fix_blk, fb.data(), (size_t)nb * sizeof(int), cudaMemcpyHostToDevice));
    }
    // segments of the vector kernels
    std::vector<int> sinst, blk0(n + 1, 0);
    std::vector<int64_t> slo, shi;
    for (int i = 0; i < n; ++i) {
        blk0[i] = (int)sinst.size();
        const int64_t nb = std::max<int64_t>(1, (b->len[i] + SEG_CHUNK - 1) / SEG_CHUNK);
        for (int64_t k = 0; k < nb; ++k) {
            sinst.push_back(i);
            slo.push_back(b->off[i] + k * SEG_CHUNK);
            shi.push_back(b->off[i] + std::min<int64_t>(b->len[i], (k + 1) * SEG_CHUNK));
        }
    }
    blk0[n] = (int)sinst.size();
    b->nblk = (int)sinst.size();
    BCK(balloc(&b->d_seg_inst, b->nblk));
    BCK(balloc(&b->d_seg_lo, b->nblk));
    BCK(balloc(&b->d_seg_hi, b->nblk));
    BCK(balloc(&b->d_blk0, n + 1));
    BCK(balloc(&b->d_len, n));
    BCK(cudaMemcpy(b->d_seg_inst, sinst.data(), b->nblk * sizeof(int), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_seg_lo, slo.data(), b->nblk * sizeof(int64_t), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_seg_hi, shi.data(), b->nblk * sizeof(int64_t), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_blk0, blk0.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_len, b->len.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
    BCK(balloc(&b->d_partial, 3 * (size_t)b->nblk));
    BCK(balloc(&b->d_active, n));
    // batch vectors (zero-filled, so that the alignment gaps between segments stay zero)
    const size_t tb = (size_t)b->total;
    for (float **p : { &b->fx, &b->fr, &b->fp, &b->fq, &b->dinv }) {
        BCK(balloc(p, tb));
        BCK(cudaMemset(*p, 0, tb * sizeof(float)));
    }
    for (double **p : { &b->R, &b->Rt, &b->B, &b->D, &b->diag }) {
        BCK(balloc(p, tb));
        BCK(cudaMemset(*p, 0, tb * sizeof(double)));
    }
    // basis pairs per order (every context of an order has the same rules)
    for (int i = 0; i < n; ++i)
        BCK(cudaMemcpyToSymbol(c_bpairs, &b->ctx[i]->p32, sizeof(BasisPairs), (b->order[i] - 1) * sizeof(BasisPairs)));
    if (b->cg_exec) { cudaGraphExecDestroy(b->cg_exec); b->cg_exec = nullptr; }
    if (b->cg_loop) { cudaGraphExecDestroy(b->cg_loop); b->cg_loop = nullptr; }
    // launch attributes and the resident CTAs per SM of this shape.  The shared-memory limit is
    // an attribute of the kernel for the whole process: raise it, never lower it below what an
    // earlier batch launches with.
    {
        static std::mutex mu;
        static size_t raised = 0;
        std::lock_guard<std::mutex> lock(mu);
        if (b->smem > raised) {
            BCK(cudaFuncSetAttribute(k_jv_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
            raised = b->smem;
        }
    }
    // policy 3: each variant's launch takes one tile's region (plus the mbarrier); raise each
    // variant kernel's limit the same way
    {
        static std::mutex mu;
        static size_t raised[NBV] = {};
        std::lock_guard<std::mutex> lock(mu);
        for (int v = 0; v < NBV; ++v) b->vsmem[v] = 0;
        for (int i = 0; i < n; ++i) {
            const int v = b->variant[i];
            b->vsmem[v] = std::max(b->vsmem[v], 64 + bv_tile_bytes(v, b->ctx[i]->tqs32));
        }
        for (int v = 0; v < NBV; ++v)
            if (b->vsmem[v] > raised[v] && b->vsmem[v] > 48 * 1024) {
                BCK(cudaFuncSetAttribute(bv_kernel(v), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->vsmem[v]));
                raised[v] = b->vsmem[v];
            }
    }
    int per_sm = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jv_batch, b->threads, b->smem));
    if (per_sm < 1) return bfail(b, FE_ERR_UNSUPPORTED, "batched launch does not fit an SM (%zu B shared)", b->smem);
    b->grid = per_sm * b->num_sms;
    return upload_work(b, b->policy);
}

fe_status setup_contexts(fe_batch *b, const fe_batch_item *items)
{
    for (fe_ctx *c : b->ctx) fe_destroy(c);
    b->ctx.assign(b->count, nullptr);
    for (int i = 0; i < b->count; ++i) {
        fe_setup_opts o{};
        o.tile = b->tile[i];
        o.per_element = 0;
        fe_status s = fe_setup_ex(items[i].mesh, items[i].order, 0, items[i].prob, &o, &b->ctx[i]);
        if (s != FE_OK) {
            char buf[64];
            std::snprintf(buf, sizeof buf, "instance %d: ", i);
            b->err = std::string(buf) + fe_last_error(nullptr);
            return s;
        }
        // the kernels index the instance's arrays by the variant's tile edge: it must be the
        // context's own
        if (b->ctx[i]->T != b->tile[i] || b->ctx[i]->k != b->order[i] || bv_of(b->order[i], b->tile[i]) != b->variant[i])
            return bfail(b, FE_ERR_STATE, "instance %d: context tile edge %d differs from the batch's %d", i,
                         b->ctx[i]->T, b->tile[i]);
    }
    return FE_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// ABI
// ------------------------------------------------------------------------------------------------
extern "C" fe_status fe_batch_create(const fe_batch_item *items, int count, const fe_batch_opts *opts, fe_batch **out)
{
    if (!out) return FE_ERR_ARG;
    *out = nullptr;
    g_batch_setup_error.clear();
    if (!items || count < 1) { g_batch_setup_error = "need at least one instance"; return FE_ERR_ARG; }
    fe_batch_opts o{};
    o.policy = -1;
    if (opts) o = *opts;
    for (int i = 0; i < count; ++i) {
        if (!items[i].mesh || !items[i].prob || items[i].mesh->dim != 3 || items[i].order < 1 ||
            items[i].order > BATCH_MAX_ORDER) {
            g_batch_setup_error = "batched instances are 3D of order 1..4";
            return items[i].order > BATCH_MAX_ORDER ? FE_ERR_UNSUPPORTED : FE_ERR_ARG;
        }
        const int *nn = items[i].mesh->n;
        if (nn[0] != nn[1] || nn[0] != nn[2] || items[i].mesh->natural_faces != 0) {
            g_batch_setup_error = "batched instances are cube lattices (n[0] = n[1] = n[2]) with every face essential";
            return FE_ERR_UNSUPPORTED;
        }
    }
    fe_batch *b = new (std::nothrow) fe_batch();
    if (!b) return FE_ERR_OOM;
    b->count = count;
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, b->device);
    const std::string gpu = prop.name;
    b->order.resize(count);
    b->tile.resize(count);
    b->variant.resize(count);
    for (int i = 0; i < count; ++i) b->order[i] = items[i].order;
    fe_status s = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) == cudaSuccess ? FE_OK : FE_ERR_CUDA;
    for (int v = 0; v < NBV && s == FE_OK; ++v)
        if (cudaStreamCreateWithFlags(&b->vst[v], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[v], cudaEventDisableTiming) != cudaSuccess)
            s = FE_ERR_CUDA;
    if (s == FE_OK && cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess) s = FE_ERR_CUDA;

    // --- tile edge per order: fixed by opts, from the cache, or measured ---
    TuneCache cache;
    const bool have_cache = cache.load(o.tune_cache);
    bool cache_dirty = false;
    int chosen[BATCH_MAX_ORDER + 1] = { 0, 0, 0, 0, 0 };
    for (int k = 1; k <= BATCH_MAX_ORDER && s == FE_OK; ++k) {
        int rep = -1;     // representative: the largest instance of order k
        for (int i = 0; i < count; ++i)
            if (b->order[i] == k && (rep < 0 || items[i].mesh->n[0] > items[rep].mesh->n[0])) rep = i;
        if (rep < 0) continue;
        const int tmax = bv_max_tile(k), tmin = bv_min_tile(k);
        if (o.tile[k - 1] > 0) {
            if (bv_of(k, o.tile[k - 1]) < 0) { s = FE_ERR_UNSUPPORTED; b->err = "tile edge not compiled for this order"; break; }
            chosen[k] = o.tile[k - 1];
            continue;
        }
        char key[256];
        std::snprintf(key, sizeof key, "%s|order%d|n%d|tile", gpu.c_str(), k, items[rep].mesh->n[0]);
        double cached = 0.0;
        if (!o.retune && have_cache && cache.get(key, &cached) && (cached == tmax || cached == tmin)) {
            chosen[k] = (int)cached;
            continue;
        }
        if (!o.tune) { chosen[k] = tmax; continue; }
        // measure the representative instance alone with both tile edges
        double best_ms = 1e300;
        for (int T : { tmax, tmin }) {
            if (T < 1 || T > items[rep].mesh->n[0]) continue;
            fe_batch one;
            one.count = 1;
            one.device = b->device;
            one.num_sms = b->num_sms;
            one.order = { k };
            one.tile = { T };
            one.variant = { bv_of(k, T) };
            one.st = b->st;
            s = setup_contexts(&one, &items[rep]);
            if (s == FE_OK) s = build_tables(&one);
            // the action's cost does not depend on the tangent's values: time it on the zero-filled
            // tangent storage (allocated by build_tables)
            double ms = 0.0;
            if (s == FE_OK) s = time_jv(&one, 10, &ms);
            if (s == FE_OK && ms < best_ms) { best_ms = ms; chosen[k] = T; }
            if (s != FE_OK && b->err.empty()) b->err = one.err;
            for (fe_ctx *c : one.ctx) fe_destroy(c);
            one.ctx.clear();
            free_batch_device(&one);
            if (one.h_state) cudaFreeHost(one.h_state);
            one.st = nullptr;
            if (s != FE_OK) break;
        }
        if (s == FE_OK) { cache.set(key, chosen[k]); cache_dirty = true; }
    }
    for (int i = 0; i < count && s == FE_OK; ++i) {
        b->tile[i] = fit_tile(b->order[i], chosen[b->order[i]], items[i].mesh->n[0]);
        if (b->tile[i] < 1) {
            s = bfail(b, FE_ERR_UNSUPPORTED, "instance %d: n = %d is below every tile edge compiled for order %d", i,
                      items[i].mesh->n[0], b->order[i]);
            break;
        }
        b->variant[i] = bv_of(b->order[i], b->tile[i]);
    }
    if (s == FE_OK) s = setup_contexts(b, items);
    if (s == FE_OK) { b->policy = o.policy >= 0 ? o.policy : 1; s = build_tables(b); }
    // --- launch shape: CTAs per SM and work order, on the whole batch (the contexts are
    //     linearised by the caller later: time the action on the zero-filled tangent storage,
    //     whose cost does not depend on the values) ---
    if (s == FE_OK && o.tune) {
        char key[256];
        uint64_t sig = 1469598103934665603ull;       // FNV-1a over (order, n, tile) of every instance
        for (int i = 0; i < count; ++i)
            for (int x : { b->order[i], items[i].mesh->n[0], b->tile[i] }) { sig ^= (uint64_t)x; sig *= 1099511628211ull; }
        std::snprintf(key, sizeof key, "%s|batch%016llx", gpu.c_str(), (unsigned long long)sig);
        double cached = 0.0;
        const int per_sm_max = b->grid / std::max(b->num_sms, 1);
        if (!o.retune && have_cache && cache.get(std::string(key) + "|grid", &cached) && cached >= 1 &&
            cached <= b->grid && cache.get(std::string(key) + "|policy", &cached)) {
            double g = 0.0;
            cache.get(std::string(key) + "|grid", &g);
            b->grid = (int)g;
            s = upload_work(b, (int)cached);
        } else {
            double best = 1e300;
            int bg = b->grid, bp = b->policy;
            std::vector<int> pols = o.policy >= 0 ? std::vector<int>{ o.policy } : std::vector<int>{ 0, 1, 2, 3 };
            for (int pol : pols) {
                // policy 3 launches one CTA per tile: the persistent grid does not apply
                for (int m = pol == 3 ? per_sm_max : 1; m <= per_sm_max && s == FE_OK; ++m) {
                    b->grid = m * b->num_sms;
                    s = upload_work(b, pol);             // the CTAs' first variants depend on the grid
                    if (s != FE_OK) break;
                    double ms = 0.0;
                    s = time_jv(b, 5, &ms);
                    if (s == FE_OK && ms < best) { best = ms; bg = b->grid; bp = pol; }
                }
            }
            b->grid = bg;
            if (s == FE_OK) s = upload_work(b, bp);
            if (s == FE_OK) {
                cache.set(std::string(key) + "|grid", bg);
                cache.set(std::string(key) + "|policy", bp);
                cache.set(std::string(key) + "|ms", best);
                cache_dirty = true;
            }
        }
    }
    if (s == FE_OK && cache_dirty && o.tune_cache) cache.save(o.tune_cache);
    if (s != FE_OK) {
        g_batch_setup_error = b->err.empty() ? "batch setup failed" : b->err;
        fe_batch_destroy(b);
        return s;
    }
    *out = b;
    return FE_OK;
}

extern "C" void fe_batch_destroy(fe_batch *b)
{
    if (!b) return;
    if (b->cg_exec) cudaGraphExecDestroy(b->cg_exec);
    if (b->cg_loop) cudaGraphExecDestroy(b->cg_loop);
    free_batch_device(b);
    if (b->h_state) cudaFreeHost(b->h_state);
    if (b->st) cudaStreamDestroy(b->st);
    for (int v = 0; v < NBV; ++v) {
        if (b->vst[v]) cudaStreamDestroy(b->vst[v]);
        if (b->join_ev[v]) cudaEventDestroy(b->join_ev[v]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (fe_ctx *c : b->ctx) fe_destroy(c);
    delete b;
}

extern "C" const char *fe_batch_last_error(const fe_batch *b)
{
    if (!b) return g_batch_setup_error.c_str();
    return b->err.c_str();
}

extern "C" fe_status fe_batch_info(const fe_batch *b, int i, int64_t *offset, int64_t *n_dofs, int *tile)
{
    if (!b || i < 0 || i >= b->count) return FE_ERR_ARG;
    if (offset) *offset = b->off[i];
    if (n_dofs) *n_dofs = b->len[i];
    if (tile) *tile = b->tile[i];
    return FE_OK;
}

extern "C" fe_status fe_batch_shape(const fe_batch *b, int64_t *total, int *grid, int *threads, int *policy,
                                    int64_t *launches)
{
    if (!b) return FE_ERR_ARG;
    if (total) *total = b->total;
    if (grid) *grid = b->grid;
    if (threads) *threads = b->threads;
    if (policy) *policy = b->policy;
    if (launches) *launches = b->launches;
    return FE_OK;
}

extern "C" fe_status fe_batch_linearize(fe_batch *b, const double *u, void *stream)
{
    if (!b || !u) return bfail(b, FE_ERR_ARG, "fe_batch_linearize: null argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < b->count; ++i) {
        fe_status s = residual_tangent32(b->ctx[i], u + b->off[i], nullptr, st);
        if (s != FE_OK) return bfail(b, s, "instance %d: %s", i, b->ctx[i]->err.c_str());
        b->launches++;
    }
    return FE_OK;
}

extern "C" fe_status fe_batch_jacobian_action(fe_batch *b, const float *v, float *y, void *stream)
{
    if (!b || !v || !y || v == y) return bfail(b, FE_ERR_ARG, "fe_batch_jacobian_action: null or aliased vectors");
    for (fe_ctx *c : b->ctx)
        if (!c->lin32) return bfail(b, FE_ERR_STATE, "no FP32 linearisation (call fe_batch_linearize)");
    return launch_jv(b, v, y, false, reinterpret_cast<cudaStream_t>(stream));
}

namespace {

void enqueue_bcg(fe_batch *b, int m, cudaStream_t st)
{
    const Seg S{ b->d_seg_inst, b->d_seg_lo, b->d_seg_hi, b->d_blk0 };
    for (int i = 0; i < m; ++i) {
        launch_jv(b, b->fp, b->fq, true, st);
        k_bcg_alpha32<<<b->nblk, SEG_THREADS, 0, st>>>(b->fp, b->fq, S, b->nblk, b->d_state, b->d_partial);
        k_bcg_update32<<<b->nblk, SEG_THREADS, 0, st>>>(b->fx, b->fr, b->fp, b->fq, b->dinv, S, b->nblk, b->d_state,
                                                        b->d_partial);
        k_bcg_direction32<<<b->nblk, SEG_THREADS, 0, st>>>(b->fp, b->fr, b->dinv, S, b->d_state);
        b->launches += 3;
    }
}

// segmented FP64 norms of vec: out[i] = ||vec_i||_2 (synchronous)
fe_status bnorms(fe_batch *b, const double *vec, std::vector<double> &out)
{
    const Seg S{ b->d_seg_inst, b->d_seg_lo, b->d_seg_hi, b->d_blk0 };
    k_bdot64<<<b->nblk, SEG_THREADS, 0, b->st>>>(vec, vec, S, b->nblk, b->d_state, b->d_partial);
    b->launches++;
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(b->h_state, b->d_state, b->count * sizeof(CgState), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    out.resize(b->count);
    for (int i = 0; i < b->count; ++i) out[i] = std::sqrt(b->h_state[i].scalar);
    return FE_OK;
}

}  // namespace

extern "C" fe_status fe_batch_newton_solve(fe_batch *b, double *u, const fe_newton_opts *opts_in,
                                           fe_newton_report *reports, fe_newton_report *total, void *stream)
{
    if (!b || !u) return bfail(b, FE_ERR_ARG, "fe_batch_newton_solve: null argument");
    fe_newton_opts o;
    if (opts_in) o = *opts_in; else fe_newton_default_opts(&o);
    const int n = b->count;
    BCK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = b->launches;
    std::vector<fe_newton_report> rep(n);
    for (auto &r : rep) std::memset(&r, 0, sizeof r);
    const Seg S{ b->d_seg_inst, b->d_seg_lo, b->d_seg_hi, b->d_blk0 };
    cudaStream_t st = b->st;
    // R and the FP32 tangent at u for every instance
    for (int i = 0; i < n; ++i) {
        fe_status s = residual_tangent32(b->ctx[i], u + b->off[i], b->R + b->off[i], st);
        if (s != FE_OK) return bfail(b, s, "instance %d: %s", i, b->ctx[i]->err.c_str());
        b->launches += 2;
    }
    std::vector<double> rn;
    BCKS(bnorms(b, b->R, rn));
    std::vector<double> r0 = rn;
    std::vector<int> active(n), status(n, FE_OK);
    for (int i = 0; i < n; ++i) {
        rep[i].r0 = r0[i];
        active[i] = std::isfinite(r0[i]) && r0[i] > 0.0;
        if (!std::isfinite(r0[i])) status[i] = FE_ERR_NAN;
    }
    double cg_ms = 0.0;
    for (int it = 0;; ++it) {
        int nact = 0;
        for (int i = 0; i < n; ++i) {
            if (active[i] && rn[i] <= o.rtol * r0[i]) active[i] = 0;
            if (active[i] && it >= o.max_newton) { active[i] = 0; status[i] = FE_ERR_NOT_CONVERGED; }
            nact += active[i];
        }
        if (nact == 0) break;
        // Jacobi scaling and right-hand side -R of the active instances
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            fe_status s = jacobi_diag32(b->ctx[i], b->diag + b->off[i], st);
            if (s != FE_OK) return bfail(b, s, "instance %d: %s", i, b->ctx[i]->err.c_str());
            b->launches += 2;
        }
        k_neg_recip<<<1216, 256, 0, st>>>(b->B, b->R, b->dinv, b->diag, b->total);
        k_bdot64<<<b->nblk, SEG_THREADS, 0, st>>>(b->B, b->B, S, b->nblk, b->d_state, b->d_partial);
        BCK(cudaMemcpyAsync(b->d_active, active.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
        k_bcg_init32<<<b->nblk, SEG_THREADS, 0, st>>>(b->B, b->dinv, b->fx, b->fr, b->fp, S, b->nblk, b->d_len,
                                                      b->d_active, b->d_state, o.cg_rtol, o.max_cg, b->d_partial);
        b->launches += 3;
        BCK(cudaGetLastError());
        // CG batches for all instances at once, replayed as one captured graph
        const auto c0 = std::chrono::steady_clock::now();
        const int m = std::max(1, o.cg_batch);
        const bool device_loop = o.use_graph == 2;
        if (device_loop && (!b->cg_loop || b->cg_loop_m != m)) {
            // a conditional WHILE node around m iterations and the condition kernel
            if (b->cg_loop) { cudaGraphExecDestroy(b->cg_loop); b->cg_loop = nullptr; }
            const int64_t lsave = b->launches;
            cudaGraph_t g = nullptr;
            BCK(cudaGraphCreate(&g, 0));
            cudaGraphConditionalHandle hc;
            BCK(cudaGraphConditionalHandleCreate(&hc, g, 1u, cudaGraphCondAssignDefault));
            cudaGraphNodeParams np = { cudaGraphNodeTypeConditional };   // aggregate: the rest zero
            np.conditional.handle = hc;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            BCK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
            cudaGraph_t body = np.conditional.phGraph_out[0];
            BCK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            enqueue_bcg(b, m, st);
            k_bcg_continue<<<1, 32, 0, st>>>(hc, b->d_state, n);
            BCK(cudaStreamEndCapture(st, &body));
            BCK(cudaGraphInstantiate(&b->cg_loop, g, 0));
            cudaGraphDestroy(g);
            b->cg_loop_m = m;
            b->launches = lsave;
        }
        if (o.use_graph == 1 && (!b->cg_exec || b->cg_batch != m)) {
            if (b->cg_exec) { cudaGraphExecDestroy(b->cg_exec); b->cg_exec = nullptr; }
            const int64_t lsave = b->launches;
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            enqueue_bcg(b, m, st);
            BCK(cudaStreamEndCapture(st, &g));
            BCK(cudaGraphInstantiate(&b->cg_exec, g, 0));
            cudaGraphDestroy(g);
            b->cg_batch = m;
            b->launches = lsave;
        }
        if (device_loop) {
            BCK(cudaGraphLaunch(b->cg_loop, st));
            BCK(cudaMemcpyAsync(b->h_state, b->d_state, n * sizeof(CgState), cudaMemcpyDeviceToHost, st));
            BCK(cudaStreamSynchronize(st));
            int maxit = 0;
            for (int i = 0; i < n; ++i) maxit = std::max(maxit, b->h_state[i].iter);
            b->launches += (int64_t)std::max(1, (maxit + m - 1) / m) * (5 * (int64_t)m + 1);
        }
        for (; !device_loop;) {
            if (o.use_graph) {
                BCK(cudaGraphLaunch(b->cg_exec, st));
                b->launches += 5 * (int64_t)m;
            } else {
                enqueue_bcg(b, m, st);
                BCK(cudaGetLastError());
            }
            BCK(cudaMemcpyAsync(b->h_state, b->d_state, n * sizeof(CgState), cudaMemcpyDeviceToHost, st));
            BCK(cudaStreamSynchronize(st));
            bool all = true;
            for (int i = 0; i < n; ++i) all = all && b->h_state[i].done != 0;
            if (all) break;
        }
        cg_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c0).count();
        int h_err = 0;
        BCK(cudaMemcpy(&h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (h_err) return bfail(b, FE_ERR_CUDA, "batched action: a bounded wait timed out (%d)", h_err);
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            const CgState &T = b->h_state[i];
            rep[i].cg_iters_total += T.iter;
            if (it < FE_NEWTON_HIST) rep[i].cg_hist[it] = T.iter;
            if (T.done == CG_BREAKDOWN || T.done == CG_NAN) {
                active[i] = 0;
                status[i] = T.done == CG_NAN ? FE_ERR_NAN : FE_ERR_BREAKDOWN;
            }
        }
        k_bcg_widen<<<b->nblk, SEG_THREADS, 0, st>>>(b->D, b->fx, S, b->d_state);
        b->launches++;
        // backtracking line search per instance, in lock step
        std::vector<double> alpha(n, 1.0);
        std::vector<int> pending = active;
        for (int h = 0; h <= o.max_halvings; ++h) {
            int np = 0;
            for (int i = 0; i < n; ++i) {
                if (!pending[i]) continue;
                ++np;
                const int64_t off = b->off[i], len = b->len[i];
                // trial point u + alpha d into B (the right-hand side is no longer needed); its
                // residual into Rt and its tangent into the instance's storage
                k_axpy_to<<<256, 256, 0, st>>>(b->B + off, u + off, alpha[i], b->D + off, len);
                fe_status s = residual_tangent32(b->ctx[i], b->B + off, b->Rt + off, st);
                if (s != FE_OK) return bfail(b, s, "instance %d: %s", i, b->ctx[i]->err.c_str());
                b->launches += 3;
            }
            if (np == 0) break;
            std::vector<double> tn;
            BCKS(bnorms(b, b->Rt, tn));
            for (int i = 0; i < n; ++i) {
                if (!pending[i]) continue;
                const bool ok = std::isfinite(tn[i]) && (!o.line_search || tn[i] <= (1.0 - o.armijo * alpha[i]) * rn[i]);
                if (ok || !o.line_search) {
                    pending[i] = 0;
                    if (!ok) { active[i] = 0; status[i] = FE_ERR_BREAKDOWN; continue; }
                    const int64_t off = b->off[i], len = b->len[i];
                    BCK(cudaMemcpyAsync(u + off, b->B + off, len * sizeof(double), cudaMemcpyDeviceToDevice, st));
                    BCK(cudaMemcpyAsync(b->R + off, b->Rt + off, len * sizeof(double), cudaMemcpyDeviceToDevice, st));
                    rn[i] = tn[i];
                    if (rep[i].newton_iters < FE_NEWTON_HIST) rep[i].r_hist[rep[i].newton_iters] = tn[i];
                    rep[i].newton_iters++;
                } else {
                    alpha[i] *= 0.5;
                    rep[i].line_search_halvings++;
                }
            }
        }
        // an accepted instance's last trial was its new point, so its stored tangent is current
        for (int i = 0; i < n; ++i)
            if (pending[i]) { active[i] = 0; status[i] = FE_ERR_BREAKDOWN; }
    }
    BCK(cudaStreamSynchronize(st));
    const double t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    fe_newton_report tot;
    std::memset(&tot, 0, sizeof tot);
    fe_status result = FE_OK;
    for (int i = 0; i < n; ++i) {
        rep[i].r_final = rn[i];
        rep[i].status = status[i];
        rep[i].t_total_ms = t_ms;
        rep[i].t_cg_ms = cg_ms;
        tot.newton_iters = std::max(tot.newton_iters, rep[i].newton_iters);
        tot.cg_iters_total += rep[i].cg_iters_total;
        tot.line_search_halvings += rep[i].line_search_halvings;
        tot.r0 += r0[i] * r0[i];
        tot.r_final += rn[i] * rn[i];
        if (status[i] != FE_OK && result == FE_OK) result = (fe_status)status[i];
    }
    tot.r0 = std::sqrt(tot.r0);
    tot.r_final = std::sqrt(tot.r_final);
    tot.t_total_ms = t_ms;
    tot.t_cg_ms = cg_ms;
    tot.kernel_launches = b->launches - l0;
    tot.status = result;
    if (reports) std::memcpy(reports, rep.data(), n * sizeof(fe_newton_report));
    if (total) *total = tot;
    if (result != FE_OK) bfail(b, result, "one or more instances did not converge (see the per-instance reports)");
    return result;
}
