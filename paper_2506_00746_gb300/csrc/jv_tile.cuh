// jv_tile.cuh -- partially assembled Jacobian action with tile-level sum factorisation (3D).
//
// y = P^T G^T B^T (T_q . B G P v) for one tile of TT^3 elements per CTA.  On a structured tile
// the element restriction G and the 1D basis operators compose into block-sparse 1D operators
//     Bt[Q1 e + q][K e + a] = B^[q][a],   Gt[Q1 e + q][K e + a] = G^[q][a]   (e < TT, a <= K),
// acting between the tile's SE = K TT + 1 DOF slots and QT = Q1 TT quadrature points per
// direction.  Sum factorisation over the tile therefore applies B G to the tile's DOF block
// directly (no per-element copies), and the transposed contractions apply G^T B^T: a DOF shared
// by two neighbouring elements of the tile receives both elements' terms, so the in-tile G^T
// needs neither staging nor atomics.  Slots on the tile's upper faces that belong to a
// neighbouring tile go to the halo buffer for the fix-up kernel.
//
// Threads: every line of a stage (e.g. the z-line of slots (sx, sy)) is split into its TT
// element segments; segment h of all lines is handled by one group of warps (packed FP32 kernel:
// thread = line + NLP * h, NLP the line count of the x stage rounded up to 32; collocated
// kernels: thread = line + lines * h with the stage's own line count, unpadded), so the lanes
// of a warp walk consecutive lines.  A transposed stage leaves the seam
// DOF between segments h and h+1 split: segment h+1's term in the array, segment h's term in a
// small seam plane; the next stage adds them (left term first).  Shared-memory strides are
// padded so that every access of a warp touches 32 distinct banks.
//
// Per CTA: one bulk copy (TMA, mbarrier-completed, bounded wait) brings the tile's stored
// tangent block into shared memory while the threads gather the DOF block.
#pragma once

#include <type_traits>

namespace feod {

__host__ __device__ constexpr inline size_t pad16(size_t b) { return (b + 15) & ~(size_t)15; }

// pad of the y-slot stride of the z/y-stage arrays that makes all their accesses bank-conflict
// free (found by exhaustive search over the access patterns of this kernel)
__host__ __device__ constexpr int tile_pad_a(int d1)
{
    return d1 == 2 ? 5 : d1 == 3 ? 8 : d1 == 4 ? 15 : d1 == 5 ? 15 : d1 == 6 ? 7 : 23;
}

template <int D1, int TT>
struct TileShape {
    static constexpr int K = D1 - 1;
    static constexpr int SE = K * TT + 1;          // DOF slots per tile edge
    static constexpr int QT = D1 * TT;             // quadrature points per tile edge
    static constexpr int NS3 = SE * SE * SE;
    static constexpr int NQT = QT * QT * QT;
    static constexpr int SA = SE * QT + tile_pad_a(D1);   // y-slot stride of A / E
    static constexpr int NA = SA * SE;             // one z- or y-stage array (A, E)
    static constexpr int NC = SE * QT * QT;        // one x-stage array (C, D)
    static constexpr int NLP = ((QT * QT + 31) / 32) * 32;   // lines per segment group
    static constexpr int THREADS = NLP * TT;
    // the collocated (FP64, double-float, residual) kernels pack each stage's lines of all
    // segments contiguously (thread = line + lines x h) where that takes fewer warps, so that a
    // stage with fewer lines than a multiple of 32 per segment leaves idle lanes only at the end:
    // every idle lane of an FP64 warp instruction is FP64-unit time lost (Colloc::line)
    static constexpr int CTHREADS = ((QT * QT * TT + 31) / 32) * 32;
    // seam planes (left terms of the DOFs shared by segments h and h+1)
    static constexpr int NSX = (TT - 1) * QT * QT; // per x-stage array
    static constexpr int NSY = (TT - 1) * QT * SE; // per y-stage array
    static constexpr int NSZ = (TT - 1) * SE * SE;
};

// Shared memory of the generic (collocated) tile kernel, in bytes from the dynamic base.  Arrays
// whose live ranges (between the kernel's barriers) do not overlap share storage:
//   Vs, the gathered DOF block (written by the prologue, read by z) lies inside C (first written
//       by y);
//   U, the values at the points (written by x1, read by x2) lies inside A (read by y, next
//       written by yT);
//   the seam planes SX, SY, SZ and S0 (written from x3 on) lie inside the tangent block Tb (last
//       read by x2).
// FX, the x-component of the flux, stays in registers: x2 and x3 map a thread to the same points.
template <int D1, int TT, typename TC, typename TIO>
struct TileLayout {
    using TS = TileShape<D1, TT>;
    static constexpr size_t A_BYTES = pad16((size_t)(TS::NA > TS::NQT ? TS::NA : TS::NQT) * sizeof(TC));
    static constexpr size_t C_BYTES = pad16((size_t)TS::NC * sizeof(TC) > (size_t)TS::NS3 * sizeof(TIO)
                                                ? (size_t)TS::NC * sizeof(TC) : (size_t)TS::NS3 * sizeof(TIO));
    static constexpr size_t SEAM_ELEMS = (size_t)TS::NSX + TS::NSY + 2 * TS::NSZ;   // SX, SY, SZ, S0
    size_t tb, codes, hd, a, c, fy, fz, total;
    __host__ __device__ explicit TileLayout(int64_t tqs)
    {
        const size_t tb_bytes = pad16((size_t)tqs * sizeof(TC));
        tb = 64;                                   // after the mbarrier
        codes = tb + (tb_bytes > SEAM_ELEMS * sizeof(TC) ? tb_bytes : pad16(SEAM_ELEMS * sizeof(TC)));
        hd = codes + pad16((size_t)TS::NS3 * 4);
        a = hd + pad16((size_t)TS::NS3 * 4);
        c = a + A_BYTES;
        fy = c + C_BYTES;
        fz = fy + pad16((size_t)TS::NQT * sizeof(TC));
        total = fz + pad16((size_t)TS::NQT * sizeof(TC));
    }
};

template <int D1, int TT, typename TC, typename TIO>
__host__ __device__ inline size_t tile_smem_bytes(int64_t tqs, int /*Spad*/)
{
    return TileLayout<D1, TT, TC, TIO>(tqs).total;
}

// n consecutive shared-memory values into registers; 16-byte vector loads when n % 4 == 0 (FP32)
// or n % 2 == 0 (8-byte types: FP64, double-float) -- the caller guarantees the alignment then.
template <int N, typename TC>
__device__ __forceinline__ void lds_run(const TC *p, TC (&r)[N])
{
    if constexpr (sizeof(TC) == 4 && N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 w = *reinterpret_cast<const float4 *>(p + i);
            r[i] = w.x; r[i + 1] = w.y; r[i + 2] = w.z; r[i + 3] = w.w;
        }
    } else if constexpr (sizeof(TC) == 8 && N % 2 == 0) {
        struct alignas(16) Two { TC a, b; };
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const Two w = *reinterpret_cast<const Two *>(p + i);
            r[i] = w.a; r[i + 1] = w.b;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = p[i];
    }
}

// Collocated stages of the generic (FP64 and double-float) tile kernel.  The forward half
// interpolates the tile's DOF block to its quadrature points (B along z, y, x), then takes the
// reference gradient there with the Q1 x Q1 collocation derivative Dc (Dc[q][j] = l_j'(x_q), l_j
// the Lagrange polynomials on the Gauss points; exact, as the interpolant has degree k = Q1 - 1
// in each direction).  The backward half applies Dc^T along x, y, z, sums, and applies B^T along
// x, y, z.  That is 12 D1^4 + 9 D1^3 multiply-adds per element, the algorithmic count, where
// carrying (B, G) pairs through the stages takes 16 D1^4 + 9 D1^3.
//
// Every stage is a function of the thread index over shared-memory arrays, run between barriers:
//   z  (line (sx, sy) of slots, segment h):  A = B_z v
//   y  (line (sx, qz)):                      C = B_y A
//   x1 (line (qy, qz)):                      U = B_x C                     (values at the points)
//   x2 (line (qy, qz)):                      g = (Dc_x U, Dc_y U, Dc_z U), f = T g -> FX, FY, FZ
//   x3 (line (qy, qz)):                      W = Dc_x^T FX + Dc_y^T FY + Dc_z^T FZ, C = B_x^T W
//   yT (line (sx, qz)):                      A = B_y^T C
//   zT (line (sx, sy)):                      out = B_z^T A, written through the slot codes
// with seam planes for the DOFs that neighbouring segments share (left term first).  In FP64 the
// z, y, yT and zT stages take one output of a line per thread instead of a line (UNITS).  The point
// arrays U, FX, FY, FZ are indexed (qx, qy, qz) -> qz + QT (qy + QT qx).  The functions are host-
// callable so that a host loop over the thread indices can run them between the same barriers.
template <int D1, int TT>
struct Colloc {
    using TS = TileShape<D1, TT>;
    static constexpr int K = TS::K, Q1 = D1, SE = TS::SE, QT = TS::QT, NQT = TS::NQT;
    static constexpr int SA = TS::SA;
    __host__ __device__ static constexpr int pidx(int qx, int qy, int qz) { return qz + QT * (qy + QT * qx); }
    // double-float: the point sums of x2 and x3 run on packed pairs at orders 3, 4 and 6 (Q1 = 4,
    // 5, 7: 7 %, 3 % and 4 % faster than with pairs only in the interpolations); at orders 1, 2
    // and 5 their extra registers cost more than the pairs save (10 %, 20 % and 2 % slower)
    static constexpr bool PK_X = Q1 == 4 || Q1 == 5 || Q1 == 7;

    // the thread mapping of a stage with NL lines per segment: thread tid takes line L of segment
    // h, tid = L + ST h, false for a thread without a line.  ST = NL (packed) where that takes
    // fewer warps than one warp-aligned group per segment; otherwise ST = NL rounded up to 32
    // (the same warps, and no lane of a warp shared by two segments)
    template <int NL>
    __host__ __device__ static bool line(int tid, int &L, int &h)
    {
        constexpr int R = (NL + 31) / 32 * 32;
        constexpr int ST = (TT * NL + 31) / 32 * 32 < TT * R ? NL : R;
        h = tid / ST;
        L = tid - ST * h;
        return h < TT && L < NL;
    }

#ifdef FEOD_F32X2
    // Double-float contractions on packed pairs of outputs: pair p holds outputs 2p and 2p + 1 (an
    // odd last output pairs with a discarded lane), and every lane runs its scalar sum's
    // operations in the scalar order, so the results are bit for bit those of the scalar code.
    template <int NP>
    __device__ static void pk_zero(df2 (&acc)[NP])
    {
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[p] = df2_zero();
    }
    // acc[p] += sum_k M[p][k] in[k] over k ascending, M a packed pair table (row stride MAXQ)
    template <int NI, int NP>
    __device__ static void pk_contract(const df2c *M, const dfloat (&in)[NI], df2 (&acc)[NP])
    {
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            const df2 x = df2_bcast(in[k]);
#pragma unroll
            for (int p = 0; p < NP; ++p) df2_fma(acc[p], M[p * MAXQ + k], x);
        }
    }
    template <int NP, int NO>
    __device__ static void pk_unpack(const df2 (&acc)[NP], dfloat (&out)[NO])
    {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            out[2 * p] = df2_lo(acc[p]);
            if (2 * p + 1 < NO) out[2 * p + 1] = df2_hi(acc[p]);
        }
    }
#endif

    // out[q] = sum_a B[q][a] in[a], each sum in ascending a; the Q1 sums advance together so that
    // their multiply-adds are independent of one another
    template <typename TC>
    __host__ __device__ static void interpolate(const BasisT<TC> &Bs, const TC (&in)[D1], TC (&out)[Q1])
    {
#ifdef FEOD_F32X2
        if constexpr (is_dfloat<TC>::value) {
            df2 acc[(Q1 + 1) / 2];
            pk_zero(acc);
            pk_contract(Bs.pk.Bq, in, acc);
            pk_unpack(acc, out);
            return;
        }
#endif
#pragma unroll
        for (int q = 0; q < Q1; ++q) out[q] = TC(0);
#pragma unroll
        for (int a = 0; a < D1; ++a)
#pragma unroll
            for (int q = 0; q < Q1; ++q) out[q] += Bs.B[q * D1 + a] * in[a];
    }

    // out[a] = sum_q B[q][a] in[q], each sum in ascending q (the transposed interpolation)
    template <typename TC>
    __host__ __device__ static void transposed(const BasisT<TC> &Bs, const TC (&in)[Q1], TC (&out)[D1])
    {
#ifdef FEOD_F32X2
        if constexpr (is_dfloat<TC>::value) {
            df2 acc[(D1 + 1) / 2];
            pk_zero(acc);
            pk_contract(Bs.pk.Bt, in, acc);
            pk_unpack(acc, out);
            return;
        }
#endif
#pragma unroll
        for (int a = 0; a < D1; ++a) out[a] = TC(0);
#pragma unroll
        for (int q = 0; q < Q1; ++q)
#pragma unroll
            for (int a = 0; a < D1; ++a) out[a] += Bs.B[q * D1 + a] * in[q];
    }

    // FP64 z, y, yT and zT stages: one output of a line per work unit (each sum in its original
    // order), the units of all segments on consecutive threads in rounds of CTHREADS.  With one
    // line per thread the last warp of a segment's lines runs its Q1 D1 multiply-adds for a few
    // lanes (order 3: 49 z-lines of a segment in two warps); FP64 instructions cost their full
    // issue whatever the lanes, so the units waste fewer (order 3: 52 + 56 + 56 + 52 instead of
    // 4 x 64 FP64 warp-instructions per tile for 49 + 56 + 56 + 49 of useful work).  The seam terms
    // of yT and zT are folded in beforehand (foldx, foldy).
    template <typename TC>
    static constexpr bool UNITS = std::is_same<TC, double>::value;

    template <typename TC, typename TIO>
    __host__ __device__ static void z(const BasisT<TC> &Bs, const TIO *Vs, TC *A, int tid)
    {
        if constexpr (UNITS<TC>) {
            // unit u = sx + SE (qq + QT sy), qq = Q1 h + q: consecutive threads, consecutive slots
            constexpr int NU = SE * QT * SE, NR = (NU + TS::CTHREADS - 1) / TS::CTHREADS;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const int u = tid + i * TS::CTHREADS;
                if (u < NU) {
                    const int sx = u % SE, w = u / SE, qq = w % QT, sy = w / QT;
                    const int h = qq / Q1, q = qq - Q1 * h;
                    TC acc = TC(0);
#pragma unroll
                    for (int a = 0; a < D1; ++a) acc += Bs.B[q * D1 + a] * (TC)Vs[((K * h + a) * SE + sy) * SE + sx];
                    A[sx + SE * qq + SA * sy] = acc;
                }
            }
            return;
        }
        int L, h;
        if (!line<SE*SE>(tid, L, h)) return;
        const int sx = L % SE, sy = L / SE;
        TC in[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) in[a] = (TC)Vs[((K * h + a) * SE + sy) * SE + sx];
        TC acc[Q1];
        interpolate(Bs, in, acc);
#pragma unroll
        for (int q = 0; q < Q1; ++q) A[sx + SE * (Q1 * h + q) + SA * sy] = acc[q];
    }

    template <typename TC>
    __host__ __device__ static void y(const BasisT<TC> &Bs, const TC *A, TC *C, int tid)
    {
        if constexpr (UNITS<TC>) {
            // unit u = (sx + SE qz) + SE QT qq, qq = Q1 h + q: the output's own index in C
            constexpr int NU = SE * QT * QT, NR = (NU + TS::CTHREADS - 1) / TS::CTHREADS;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const int u = tid + i * TS::CTHREADS;
                if (u < NU) {
                    const int xz = u % (SE * QT), qq = u / (SE * QT);
                    const int h = qq / Q1, q = qq - Q1 * h;
                    TC acc = TC(0);
#pragma unroll
                    for (int a = 0; a < D1; ++a) acc += Bs.B[q * D1 + a] * A[xz + SA * (K * h + a)];
                    C[u] = acc;
                }
            }
            return;
        }
        int L, h;
        if (!line<SE*QT>(tid, L, h)) return;
        const int sx = L % SE, qz = L / SE;
        TC in[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) in[a] = A[sx + SE * qz + SA * (K * h + a)];
        TC acc[Q1];
        interpolate(Bs, in, acc);
#pragma unroll
        for (int q = 0; q < Q1; ++q) C[sx + SE * qz + SE * QT * (Q1 * h + q)] = acc[q];
    }

    template <typename TC>
    __host__ __device__ static void x1(const BasisT<TC> &Bs, const TC *C, TC *U, int tid)
    {
        int L, h;
        if (!line<QT*QT>(tid, L, h)) return;
        const int qz = L % QT, qy = L / QT;
        const int xo = SE * qz + SE * QT * qy + K * h;
        TC in[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) in[a] = C[xo + a];
        TC acc[Q1];
        interpolate(Bs, in, acc);
#pragma unroll
        for (int q = 0; q < Q1; ++q) U[pidx(Q1 * h + q, qy, qz)] = acc[q];
    }

    // Tb: the tile's tangent block, layout [6][ex][qy][qz][qx] (qx element-local), components
    // xx yy zz xy xz yz of the symmetric dq/dg
    // fx: this thread's x-flux at its Q1 points (registers in the kernel), read back by x3
    template <typename TC>
    __host__ __device__ static void x2(const BasisT<TC> &Bs, const TC *Tb, const TC *U, TC *fx, TC *FY, TC *FZ,
                                       int tid)
    {
        int L, h;
        if (!line<QT*QT>(tid, L, h)) return;
        const int qz = L % QT, qy = L / QT;
        const int y0 = Q1 * (qy / Q1), yl = qy % Q1, z0 = Q1 * (qz / Q1), zl = qz % Q1;
        const TC *Tl = Tb + Q1 * (qz + QT * (qy + QT * h));
        TC u[Q1];
#pragma unroll
        for (int j = 0; j < Q1; ++j) u[j] = U[pidx(Q1 * h + j, qy, qz)];
#ifdef FEOD_F32X2
        if constexpr (is_dfloat<TC>::value && PK_X) {
            // the points in pairs (q, q + 1): gradient sums, then the flux, lane by lane as below
            constexpr int NP = (Q1 + 1) / 2;
            df2 gx[NP], gy[NP], gz[NP];
            pk_zero(gx); pk_zero(gy); pk_zero(gz);
#pragma unroll
            for (int j = 0; j < Q1; ++j) {
                const df2 uj = df2_bcast(u[j]);
                const df2c cy = df2c_bcast(Bs.Dc[yl * Q1 + j]), cz = df2c_bcast(Bs.Dc[zl * Q1 + j]);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int qa = Q1 * h + 2 * p, qb = 2 * p + 1 < Q1 ? qa + 1 : qa;
                    df2_fma(gx[p], Bs.pk.Dq[p * MAXQ + j], uj);
                    df2_fma(gy[p], cy, df2_pack(U[pidx(qa, y0 + j, qz)], U[pidx(qb, y0 + j, qz)]));
                    df2_fma(gz[p], cz, df2_pack(U[pidx(qa, qy, z0 + j)], U[pidx(qb, qy, z0 + j)]));
                }
            }
            const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int q0 = 2 * p, q1 = 2 * p + 1 < Q1 ? q0 + 1 : q0;
                df2 t[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) t[c] = df2_pack(Tl[c * NQT + q0], Tl[c * NQT + q1]);
                const float2 ngx = __fmul2_rn(gx[p].h, m1), ngy = __fmul2_rn(gy[p].h, m1),
                             ngz = __fmul2_rn(gz[p].h, m1);
                // t: xx yy zz xy xz yz
                auto row = [&](const df2 &ta, const df2 &tb, const df2 &tc) {
                    const dprod2 a = df2_mul(ta, gx[p], ngx), b = df2_mul(tb, gy[p], ngy),
                                 c = df2_mul(tc, gz[p], ngz);
                    const df2 ab = df2_add(a.p, a.e, b.p, b.e);
                    return df2_add(ab.h, ab.l, c.p, c.e);
                };
                const df2 f0 = row(t[0], t[3], t[4]), f1 = row(t[3], t[1], t[5]), f2 = row(t[4], t[5], t[2]);
                const int qx = Q1 * h + q0;
                fx[q0] = df2_lo(f0);
                FY[pidx(qx, qy, qz)] = df2_lo(f1);
                FZ[pidx(qx, qy, qz)] = df2_lo(f2);
                if (2 * p + 1 < Q1) {
                    fx[q0 + 1] = df2_hi(f0);
                    FY[pidx(qx + 1, qy, qz)] = df2_hi(f1);
                    FZ[pidx(qx + 1, qy, qz)] = df2_hi(f2);
                }
            }
            return;
        }
#endif
        // the 3 Q1 gradient sums (each in ascending j) advance together
        TC gxs[Q1], gys[Q1], gzs[Q1];
#pragma unroll
        for (int q = 0; q < Q1; ++q) { gxs[q] = TC(0); gys[q] = TC(0); gzs[q] = TC(0); }
#pragma unroll
        for (int j = 0; j < Q1; ++j)
#pragma unroll
            for (int q = 0; q < Q1; ++q) {
                const int qx = Q1 * h + q;
                gxs[q] += Bs.Dc[q * Q1 + j] * u[j];
                gys[q] += Bs.Dc[yl * Q1 + j] * U[pidx(qx, y0 + j, qz)];
                gzs[q] += Bs.Dc[zl * Q1 + j] * U[pidx(qx, qy, z0 + j)];
            }
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            const int qx = Q1 * h + q;
            const TC gx = gxs[q], gy = gys[q], gz = gzs[q];
            const TC txx = Tl[q], tyy = Tl[NQT + q], tzz = Tl[2 * NQT + q];
            const TC txy = Tl[3 * NQT + q], txz = Tl[4 * NQT + q], tyz = Tl[5 * NQT + q];
            fx[q] = txx * gx + txy * gy + txz * gz;
            FY[pidx(qx, qy, qz)] = txy * gx + tyy * gy + tyz * gz;
            FZ[pidx(qx, qy, qz)] = txz * gx + tyz * gy + tzz * gz;
        }
    }

    template <typename TC>
    __host__ __device__ static void x3(const BasisT<TC> &Bs, const TC *fx, const TC *FY, const TC *FZ, TC *C,
                                       TC *SX, int tid)
    {
        x3s<TC, false>(Bs, fx, fx, FY, FZ, C, SX, tid);
    }

    // x3 with (HAS_S) a value term s at this thread's Q1 points: W = Dc^T F + s before B_x^T (the
    // residual's load term); without it the sums start from zero
    template <typename TC, bool HAS_S>
    __host__ __device__ static void x3s(const BasisT<TC> &Bs, const TC *fx, const TC *s, const TC *FY,
                                        const TC *FZ, TC *C, TC *SX, int tid)
    {
        int L, h;
        if (!line<QT*QT>(tid, L, h)) return;
        const int qz = L % QT, qy = L / QT;
        const int y0 = Q1 * (qy / Q1), yl = qy % Q1, z0 = Q1 * (qz / Q1), zl = qz % Q1;
        const int xo = SE * qz + SE * QT * qy + K * h;
#ifdef FEOD_F32X2
        if constexpr (is_dfloat<TC>::value && PK_X) {
            // W in pairs of points (q, q + 1), lane by lane as below
            constexpr int NP = (Q1 + 1) / 2;
            df2 wp[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                if constexpr (HAS_S) wp[p] = df2_pack(s[2 * p], s[2 * p + 1 < Q1 ? 2 * p + 1 : 2 * p]);
                else wp[p] = df2_zero();
            }
#pragma unroll
            for (int j = 0; j < Q1; ++j) {
                const df2 fj = df2_bcast(fx[j]);
                const df2c cy = df2c_bcast(Bs.Dc[j * Q1 + yl]), cz = df2c_bcast(Bs.Dc[j * Q1 + zl]);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const int qa = Q1 * h + 2 * p, qb = 2 * p + 1 < Q1 ? qa + 1 : qa;
                    df2_fma(wp[p], Bs.pk.Dt[p * MAXQ + j], fj);
                    df2_fma(wp[p], cy, df2_pack(FY[pidx(qa, y0 + j, qz)], FY[pidx(qb, y0 + j, qz)]));
                    df2_fma(wp[p], cz, df2_pack(FZ[pidx(qa, qy, z0 + j)], FZ[pidx(qb, qy, z0 + j)]));
                }
            }
            TC w[Q1], d[D1];
            pk_unpack(wp, w);
            transposed(Bs, w, d);
#pragma unroll
            for (int a = 0; a < K; ++a) C[xo + a] = d[a];
            if (h == TT - 1) C[xo + K] = d[K];
            else SX[h * QT * QT + L] = d[K];
            return;
        }
#endif
        // the Q1 sums W[q] (each over j ascending, x then y then z term) advance together
        TC w[Q1];
#pragma unroll
        for (int q = 0; q < Q1; ++q) w[q] = HAS_S ? s[q] : TC(0);
#pragma unroll
        for (int j = 0; j < Q1; ++j)
#pragma unroll
            for (int q = 0; q < Q1; ++q) {
                const int qx = Q1 * h + q;
                w[q] += Bs.Dc[j * Q1 + q] * fx[j];
                w[q] += Bs.Dc[j * Q1 + yl] * FY[pidx(qx, y0 + j, qz)];
                w[q] += Bs.Dc[j * Q1 + zl] * FZ[pidx(qx, qy, z0 + j)];
            }
        TC d[D1];
        transposed(Bs, w, d);
#pragma unroll
        for (int a = 0; a < K; ++a) C[xo + a] = d[a];
        if (h == TT - 1) C[xo + K] = d[K];
        else SX[h * QT * QT + L] = d[K];
    }

    // FP64 backward half: the seam terms are added once, in place, before the stage that reads
    // them (the units of yT and zT then run without a branch that every warp would issue): C at
    // the x-seam slots sx = K m gets SX (left term first, as yT adds it), after x3; A at the y-seam
    // slots gets SY, after yT.
    template <typename TC>
    __host__ __device__ static void foldx(TC *C, const TC *SX, int tid)
    {
        constexpr int NU = TS::NSX, NR = (NU + TS::CTHREADS - 1) / TS::CTHREADS;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int u = tid + i * TS::CTHREADS;       // u = qz + QT qy + QT QT (m - 1)
            if (u < NU) {
                const int qzy = u % (QT * QT), m = u / (QT * QT) + 1, qz = qzy % QT, qy = qzy / QT;
                TC &c = C[K * m + SE * qz + SE * QT * qy];
                c = SX[u] + c;
            }
        }
    }
    template <typename TC>
    __host__ __device__ static void foldy(TC *A, const TC *SY, int tid)
    {
        constexpr int NU = TS::NSY, NR = (NU + TS::CTHREADS - 1) / TS::CTHREADS;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int u = tid + i * TS::CTHREADS;       // u = zx + SE qz + SE QT (m - 1)
            if (u < NU) {
                const int xz = u % (SE * QT), m = u / (SE * QT) + 1;
                TC &a = A[xz + SA * (K * m)];
                a = SY[u] + a;
            }
        }
    }

    // U: the unit mapping (the caller has run foldx), else one line per thread with the seam
    // terms added here
    template <typename TC, bool U = UNITS<TC>>
    __host__ __device__ static void yT(const BasisT<TC> &Bs, const TC *C, const TC *SX, TC *A, TC *SY, int tid)
    {
        if constexpr (U) {
            // one output node a of a line per unit (C's x-seams folded in by foldx), unit
            // u = xz + SE QT (a + D1 h), xz = sx + SE qz
            constexpr int NU = SE * QT * D1 * TT, NR = (NU + TS::CTHREADS - 1) / TS::CTHREADS;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const int u = tid + i * TS::CTHREADS;
                if (u < NU) {
                    const int xz = u % (SE * QT), w = u / (SE * QT), a = w % D1, h = w / D1;
                    TC acc = TC(0);
#pragma unroll
                    for (int q = 0; q < Q1; ++q) acc += Bs.B[q * D1 + a] * C[xz + SE * QT * (Q1 * h + q)];
                    if (a < K) A[xz + SA * (K * h + a)] = acc;
                    else if (h == TT - 1) A[xz + SA * (SE - 1)] = acc;
                    else SY[h * QT * SE + xz] = acc;
                }
            }
            return;
        }
        int L, h;
        if (!line<SE*QT>(tid, L, h)) return;
        const int sx = L % SE, qz = L / SE;
        const bool xseam = (sx % K == 0) && sx > 0 && sx < SE - 1;
        TC e[Q1];
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            const int qy = Q1 * h + q;
            e[q] = C[sx + SE * qz + SE * QT * qy];
            if (xseam) e[q] = SX[(sx / K - 1) * QT * QT + qz + QT * qy] + e[q];
        }
        TC E[D1];
        transposed(Bs, e, E);
#pragma unroll
        for (int a = 0; a < K; ++a) A[sx + SE * qz + SA * (K * h + a)] = E[a];
        if (h == TT - 1) A[sx + SE * qz + SA * (SE - 1)] = E[K];
        else SY[h * QT * SE + L] = E[K];
    }

    // out0: this thread's term of slot K h, added by seam() after the next barrier (h > 0)
    template <typename TC, typename W, bool U = UNITS<TC>>
    __host__ __device__ static void zT(const BasisT<TC> &Bs, const TC *A, const TC *SY, TC *SZ, const W &write,
                                       TC &out0, int tid)
    {
        if constexpr (U) {
            // one output node a of a line per unit (A's y-seams folded in by foldy), unit
            // u = L + SE SE (a + D1 h), L = zx + SE zy; node 0 of segment h > 0 goes to the plane
            // S0 = SZ + NSZ for seam()
            constexpr int NU = SE * SE * D1 * TT, NR = (NU + TS::CTHREADS - 1) / TS::CTHREADS;
            TC *S0 = SZ + TS::NSZ;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const int u = tid + i * TS::CTHREADS;
                if (u < NU) {
                    const int L = u % (SE * SE), w = u / (SE * SE), a = w % D1, h = w / D1;
                    const int zx = L % SE, zy = L / SE;
                    TC acc = TC(0);
#pragma unroll
                    for (int q = 0; q < Q1; ++q) acc += Bs.B[q * D1 + a] * A[zx + SE * (Q1 * h + q) + SA * zy];
                    if (a > 0 && a < K) write((K * h + a) * SE * SE + L, acc);
                    else if (a == 0) {
                        if (h == 0) write(L, acc);
                        else S0[(h - 1) * SE * SE + L] = acc;
                    } else if (h == TT - 1) write((SE - 1) * SE * SE + L, acc);
                    else SZ[h * SE * SE + L] = acc;
                }
            }
            return;
        }
        int L, h;
        if (!line<SE*SE>(tid, L, h)) return;
        const int zx = L % SE, zy = L / SE;
        const bool yseam = (zy % K == 0) && zy > 0 && zy < SE - 1;
        TC zv[Q1];
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            const int qz = Q1 * h + q;
            zv[q] = A[zx + SE * qz + SA * zy];
            if (yseam) zv[q] = SY[(zy / K - 1) * QT * SE + zx + SE * qz] + zv[q];
        }
        TC out[D1];
        transposed(Bs, zv, out);
        const int s0 = zy * SE + zx;
#pragma unroll
        for (int a = 1; a < K; ++a) write((K * h + a) * SE * SE + s0, out[a]);
        if (h == 0) write(s0, out[0]);
        if (h == TT - 1) write((SE - 1) * SE * SE + s0, out[K]);
        else SZ[h * SE * SE + L] = out[K];
        out0 = out[0];
    }

    template <typename TC, typename W, bool U = UNITS<TC>>
    __host__ __device__ static void seam(const TC *SZ, const W &write, TC out0, int tid)
    {
        if constexpr (U) {
            constexpr int NU = SE * SE * (TT - 1), NR = (NU + TS::CTHREADS - 1) / TS::CTHREADS;
            const TC *S0 = SZ + TS::NSZ;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const int u = tid + i * TS::CTHREADS;
                if (u < NU) write((K * (u / (SE * SE) + 1)) * SE * SE + u % (SE * SE), SZ[u] + S0[u]);
            }
            return;
        }
        int L, h;
        if (!line<SE * SE>(tid, L, h) || h == 0) return;
        write((K * h * SE + L / SE) * SE + L % SE, SZ[(h - 1) * SE * SE + L] + out0);
    }
};

// The writes of one tile: P^T (essential rows: J v = v), the halo partial sums of slots that a
// neighbouring tile owns, the tile's own DOFs.
template <typename TC, typename TIO>
struct SlotWriter {
    const uint32_t *codes, *hd;
    const TIO *v;
    TIO *y;
    TC *halo;
    __host__ __device__ void operator()(int s, TC val) const
    {
        const uint32_t code = codes[s];
        if (code == SLOT_INVALID) return;
        const uint32_t g = code & SLOT_GMASK;
        if (code & SLOT_HALO) {
            if (!(code & SLOT_ESS)) halo[hd[s]] = val;
        } else if (code & SLOT_ESS) {
            y[g] = v[g];
        } else {
            y[g] = (TIO)val;
        }
    }
};

// One CTA per tile.  Thread 0 starts the bulk copy of the tile's tangent block; meanwhile all
// threads load the slot codes, then (in one batch) the input values and, for halo slots, their
// halo-array positions.
// small CTAs (one-element tiles of high order) get a register budget that leaves room for
// several CTAs per SM: at most 128 registers per thread
template <int THREADS>
constexpr int tile_min_blocks() { return THREADS <= 128 ? 512 / THREADS : 1; }

template <int D1, int TT, typename TC, typename TIO>
__global__ void __launch_bounds__(TileShape<D1, TT>::CTHREADS, tile_min_blocks<TileShape<D1, TT>::CTHREADS>())
    k_jv_tile(const __grid_constant__ OpParams P, const __grid_constant__ BasisT<TC> Bs, const TC *__restrict__ Tq,
              const TIO *__restrict__ v, TIO *__restrict__ y, TC *__restrict__ halo)
{
    using TS = TileShape<D1, TT>;
    using S = Colloc<D1, TT>;
    constexpr int NS3 = TS::NS3, NSX = TS::NSX, NSY = TS::NSY;
    constexpr int NTH = TS::CTHREADS;
    if (P.skip && *P.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t t = P.t0 + blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t tqs = tq_stride<TC>(P);
    const uint32_t tq_bytes = (uint32_t)(tqs * sizeof(TC));

    const TileLayout<D1, TT, TC, TIO> lay(tqs);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    TC *Tb = reinterpret_cast<TC *>(smem + lay.tb);
    uint32_t *codes = reinterpret_cast<uint32_t *>(smem + lay.codes);
    uint32_t *hd = reinterpret_cast<uint32_t *>(smem + lay.hd);
    TC *A = reinterpret_cast<TC *>(smem + lay.a);
    TC *U = A;                                          // x1 .. x2
    TC *C = reinterpret_cast<TC *>(smem + lay.c);
    TIO *Vs = reinterpret_cast<TIO *>(smem + lay.c);    // prologue .. z
    TC *FY = reinterpret_cast<TC *>(smem + lay.fy);
    TC *FZ = reinterpret_cast<TC *>(smem + lay.fz);
    TC *SX = Tb;                                        // x3 .. seam
    TC *SY = SX + NSX;
    TC *SZ = SY + NSY;

    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(mbar, tq_bytes);
        tma_load_1d(Tb, Tq + t * tqs, tq_bytes, mbar);
    }
    {
        constexpr int NPER = (NS3 + NTH - 1) / NTH;
        const uint32_t *sl = P.slot + t * P.Spad;
        const uint32_t *hs = P.hdst + t * P.Spad;
        uint32_t cr[NPER], hr[NPER];
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            cr[i] = s < NS3 ? sl[s] : SLOT_INVALID;
        }
        TIO vr[NPER];
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            vr[i] = (cr[i] & SLOT_ESS) ? TIO(0) : v[cr[i] & SLOT_GMASK];
            hr[i] = (cr[i] & SLOT_HALO) && !(cr[i] & SLOT_ESS) ? hs[tid + i * NTH] : 0u;
        }
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            if (s < NS3) { codes[s] = cr[i]; Vs[s] = vr[i]; hd[s] = hr[i]; }
        }
    }
    // makes thread 0's mbarrier initialisation (and the gathered block) visible before any thread
    // polls the barrier
    __syncthreads();
    // the tangent block must have landed (bounded wait; uniform decision)
    if (__syncthreads_or(!mbar_wait_bounded(mbar, 0))) {
        if (tid == 0) {
            atomicExch(P.err, 3);
            mbar_wait_bounded(mbar, 0);
        }
        return;
    }
    const SlotWriter<TC, TIO> write{ codes, hd, v, y, halo };
    TC out0 = TC(0);
    S::z(Bs, Vs, A, tid);
    __syncthreads();
    S::y(Bs, A, C, tid);
    __syncthreads();
    S::x1(Bs, C, U, tid);
    __syncthreads();
    TC fx[D1];
    S::x2(Bs, Tb, U, fx, FY, FZ, tid);
    __syncthreads();
    S::x3(Bs, fx, FY, FZ, C, SX, tid);
    __syncthreads();
    if constexpr (S::template UNITS<TC>) {
        S::foldx(C, SX, tid);
        __syncthreads();
    }
    S::yT(Bs, C, SX, A, SY, tid);
    __syncthreads();
    if constexpr (S::template UNITS<TC>) {
        S::foldy(A, SY, tid);
        __syncthreads();
    }
    S::zT(Bs, A, SY, SZ, write, out0, tid);
    __syncthreads();
    S::seam(SZ, write, out0, tid);
}

// ------------------------------------------------------------------------------------------------
// FP32 variant with packed two-lane arithmetic
// ------------------------------------------------------------------------------------------------
// The same stages, with the contraction arrays carried as pairs so that one packed FP32
// multiply-add (FFMA2) and one 64-bit shared-memory access serve two of them:
//   after z   : (B_z v, G_z v)                            pair array A2
//   after y   : c00 = B_y B_z v scalar (C1), (G_y B_z v, B_y G_z v) pair (C2)
//   x         : gradient (G c00 | B (c01, c10)), D, transpose into d00 (C1) and (d01, d10) (C2)
//   after y^T : (E0, E1) pair (A2 again), E0 = B^T d00 + G^T d01, E1 = B^T d10
//   z^T       : (B^T E0, G^T E1) pair, summed at the end
// Pair arrays use a y-slot stride congruent to SE mod 16, so that every half-warp's 64-bit access
// touches 16 distinct bank pairs; the x stage's accesses have lane stride SE (odd) and are
// conflict-free in both widths.
// Shared-memory lifetimes let two regions double up: the gathered input block (read only by the
// z stage) lives inside the x-stage pair array C2 (first written by the y stage), and the seam
// planes (written from the x stage's end on) live inside the tangent buffer, which the x stage
// has finished reading by then.
//
// The slot codes and halo positions are read twice: by the gather (codes, into registers) and by
// the writes of the last stage.  The writes either read them from shared memory, where the
// prologue stored them, or -- "late codes" -- load their own slots' entries from global memory
// at the start of the y^T stage (the gather read the same lines a few microseconds earlier, so
// they are L2 hits, and the y^T and z^T contractions cover the latency).  Late codes free
// 2 x NS3 words of shared memory per tile and cost those loads; a variant takes them where the
// smaller footprint raises the CTAs per SM that shared memory allows (GB300: 228 KB per SM,
// 1 KB reserved per CTA, at most 2048 threads and 32 CTAs per SM): orders 3-6 of the
// single-instance kernel (9 -> 10, 4 -> 5, 2 -> 3 and 12 -> 14 CTAs per SM), not orders 1-2.
__host__ __device__ constexpr int tile2_ctas_per_sm(size_t smem_bytes, int threads)
{
    const int by_smem = (int)((size_t)228 * 1024 / (smem_bytes + 1024));
    const int by_threads = 2048 / threads;
    return by_smem < by_threads ? (by_smem < 32 ? by_smem : 32) : (by_threads < 32 ? by_threads : 32);
}

template <int D1, int TT>
struct TileShape2 : TileShape<D1, TT> {
    using B = TileShape<D1, TT>;
    static constexpr int SA2 = B::SE * B::QT + (((B::SE - B::SE * B::QT) % 16) + 16) % 16;
    static constexpr int NA2 = SA2 * B::SE;
    static constexpr size_t SEAM_BYTES = pad16((size_t)B::NSX * 4) + pad16((size_t)B::NSX * 8) +
                                         pad16((size_t)B::NSY * 8) + pad16((size_t)B::NSZ * 4);
    static constexpr size_t TANGENT_MIN_BYTES = (size_t)6 * TT * TT * TT * D1 * D1 * D1 * 4;
    static constexpr size_t CODES_BYTES = 2 * pad16((size_t)B::NS3 * 4);   // slot codes + halo positions
    static constexpr size_t CORE_BYTES = 64 + pad16(TANGENT_MIN_BYTES) + pad16((size_t)NA2 * 8) +
                                         pad16((size_t)B::NC * 4) + pad16((size_t)B::NC * 8);
    static constexpr bool LATE_CODES = tile2_ctas_per_sm(CORE_BYTES, B::THREADS) >
                                       tile2_ctas_per_sm(CORE_BYTES + CODES_BYTES, B::THREADS);
};

template <int D1, int TT, typename TIO>
__host__ __device__ inline size_t tile2_smem_bytes(int64_t tqs)
{
    using TS = TileShape2<D1, TT>;
    static_assert(TS::SEAM_BYTES <= TS::TANGENT_MIN_BYTES, "seam planes must fit in the tangent buffer");
    static_assert((size_t)TS::NS3 * 8 <= (size_t)TS::NC * 8, "the input block must fit in C2");
    return 64 + pad16((size_t)tqs * 4) + (TS::LATE_CODES ? 0 : TS::CODES_BYTES) + pad16((size_t)TS::NA2 * 8) +
           pad16((size_t)TS::NC * 4) + pad16((size_t)TS::NC * 8);
}

// Barrier policies of the packed tile code: the whole CTA, or one named barrier over a group of
// threads (a CTA that runs several tiles at once, each on its own thread group).
struct CtaBar {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
};
struct GroupBar {
    int id, count;      // barrier 1..15 (0 is __syncthreads'), threads (a multiple of 32)
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory"); }
    __device__ __forceinline__ bool any(bool p) const
    {
        int r;
        asm volatile("{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, %2, %3, pi;\n\t"
                     "selp.u32 %0, 1, 0, po;\n\t}"
                     : "=r"(r) : "r"((int)p), "r"(id), "r"(count) : "memory");
        return r != 0;
    }
};

// codes, hd: the tile's slot codes and halo positions, in shared memory or (late codes) in
// global memory.  store_hd() runs after the z stage: it stores the halo positions that the
// prologue loaded into registers (shared-memory codes only; their latency overlaps the z stage).
// tangent_ready() runs in every thread before the x stage (the first reader of Tb) and returns
// false, uniformly, to abandon the tile.
// vess: the source of the essential rows' output (J v = v there), v itself unless the output type
// differs from the input type.
template <int D1, int TT, typename TIO, typename TOUT, typename Bar, typename StoreHd, typename Ready>
__device__ __forceinline__ bool tile_stages2(const BasisPairs &Pr, const float *Tb, const TIO *Vs,
                                             const uint32_t *__restrict__ codes, const uint32_t *__restrict__ hd,
                                             float2 *A2, float *C1,
                                             float2 *C2, float *SX1, float2 *SX2, float2 *SY2, float *SZ1,
                                             const TOUT *__restrict__ vess, TOUT *__restrict__ y,
                                             float *__restrict__ halo, int tid, const Bar &bar,
                                             StoreHd store_hd, Ready tangent_ready)
{
    using TS = TileShape2<D1, TT>;
    constexpr int K = TS::K, Q1 = D1, SE = TS::SE, QT = TS::QT, NQT = TS::NQT;
    constexpr int SA2 = TS::SA2, NLP = TS::NLP;
    const int L = tid % NLP, h = tid / NLP;
    const bool live = h < TT;      // threads past the variant's count only take part in barriers

    // z: segment h of line (sx, sy): (B v, G v) at Q1 points
    if (live && L < SE * SE) {
        const int sx = L % SE, sy = L / SE;
        float in[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) in[a] = (float)Vs[((K * h + a) * SE + sy) * SE + sx];
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < D1; ++a) acc = __ffma2_rn(Pr.BG[q * D1 + a], make_float2(in[a], in[a]), acc);
            A2[sx + SE * (Q1 * h + q) + SA2 * sy] = acc;
        }
    }
    store_hd();
    bar.sync();
    // y: segment h of line (sx, qz)
    if (live && L < SE * QT) {
        const int sx = L % SE, qz = L / SE;
        float2 a2[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) a2[a] = A2[sx + SE * qz + SA2 * (K * h + a)];
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            float c00 = 0.f;
            float2 cp = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < D1; ++a) {
                c00 = fmaf(Pr.BG[q * D1 + a].x, a2[a].x, c00);
                cp = __ffma2_rn(Pr.GB[q * D1 + a], a2[a], cp);
            }
            const int o = sx + SE * qz + SE * QT * (Q1 * h + q);
            C1[o] = c00;
            C2[o] = cp;
        }
    }
    bar.sync();
    // x: segment h of line (qy, qz): gradient, D, x transpose
    if (!tangent_ready()) return false;
    float d00[D1];
    float2 dp[D1];
    const bool actx = live && L < QT * QT;
    const int xqz = L % QT, xqy = L / QT;
    const int xo = SE * xqz + SE * QT * xqy + K * h;
    if (actx) {
        float c00[D1];
        float2 cp[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) {
            c00[a] = C1[xo + a]; cp[a] = C2[xo + a];
            d00[a] = 0.f; dp[a] = make_float2(0.f, 0.f);
        }
        const float *Tl = Tb + Q1 * (xqz + QT * (xqy + QT * h));
        float txx[Q1], tyy[Q1], tzz[Q1], txy[Q1], txz[Q1], tyz[Q1];
        lds_run<Q1, float>(Tl, txx);
        lds_run<Q1, float>(Tl + NQT, tyy);
        lds_run<Q1, float>(Tl + 2 * NQT, tzz);
        lds_run<Q1, float>(Tl + 3 * NQT, txy);
        lds_run<Q1, float>(Tl + 4 * NQT, txz);
        lds_run<Q1, float>(Tl + 5 * NQT, tyz);
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            float gx = 0.f;
            float2 gyz = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < D1; ++a) {
                gx = fmaf(Pr.GB[q * D1 + a].x, c00[a], gx);
                gyz = __ffma2_rn(Pr.BB[q * D1 + a], cp[a], gyz);
            }
            const float fx = txx[q] * gx + txy[q] * gyz.x + txz[q] * gyz.y;
            float2 fyz = __fmul2_rn(make_float2(txy[q], txz[q]), make_float2(gx, gx));
            fyz = __ffma2_rn(make_float2(tyy[q], tyz[q]), make_float2(gyz.x, gyz.x), fyz);
            fyz = __ffma2_rn(make_float2(tyz[q], tzz[q]), make_float2(gyz.y, gyz.y), fyz);
#pragma unroll
            for (int a = 0; a < D1; ++a) {
                d00[a] = fmaf(Pr.GB[q * D1 + a].x, fx, d00[a]);
                dp[a] = __ffma2_rn(Pr.BB[q * D1 + a], fyz, dp[a]);
            }
        }
    }
    bar.sync();       // every segment has read its c values before any is overwritten
    if (actx) {
#pragma unroll
        for (int a = 0; a < K; ++a) { C1[xo + a] = d00[a]; C2[xo + a] = dp[a]; }
        if (h == TT - 1) {
            C1[xo + K] = d00[K]; C2[xo + K] = dp[K];
        } else {
            const int so = h * QT * QT + L;
            SX1[so] = d00[K]; SX2[so] = dp[K];
        }
    }
    bar.sync();
    // the z^T stage's slots: segment h of line (zx, zy); late codes are loaded here
    const bool actz = live && L < SE * SE;
    const int zx = L % SE, zy = L / SE;
    uint32_t zc[D1], zh[D1];
    if constexpr (TS::LATE_CODES) {
        if (actz) {
#pragma unroll
            for (int a = 0; a < D1; ++a) {
                const int s = ((K * h + a) * SE + zy) * SE + zx;
                zc[a] = codes[s];
                zh[a] = hd[s];
            }
        }
    }
    // y transpose: segment h of line (sx, qz)
    if (live && L < SE * QT) {
        const int sx = L % SE, qz = L / SE;
        const bool xseam = (sx % K == 0) && sx > 0 && sx < SE - 1;
        float e00[Q1];
        float2 ep[Q1];
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            const int qy = Q1 * h + q;
            const int o = sx + SE * qz + SE * QT * qy;
            e00[q] = C1[o]; ep[q] = C2[o];
            if (xseam) {
                const int so = (sx / K - 1) * QT * QT + qz + QT * qy;
                e00[q] = SX1[so] + e00[q];
                ep[q] = __fadd2_rn(SX2[so], ep[q]);
            }
        }
        float2 E[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) E[a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < Q1; ++q)
#pragma unroll
            for (int a = 0; a < D1; ++a) {
                E[a] = __ffma2_rn(Pr.GB[q * D1 + a], ep[q], E[a]);
                E[a].x = fmaf(Pr.BG[q * D1 + a].x, e00[q], E[a].x);
            }
#pragma unroll
        for (int a = 0; a < K; ++a) A2[sx + SE * qz + SA2 * (K * h + a)] = E[a];
        if (h == TT - 1) A2[sx + SE * qz + SA2 * (SE - 1)] = E[K];
        else SY2[h * QT * SE + L] = E[K];
    }
    bar.sync();
    // z transpose: segment h of line (zx, zy); P^T and the writes (slot a of the segment)
    float out[D1];
    auto write_slot = [&](int a, float val) {
        const int s = ((K * h + a) * SE + zy) * SE + zx;
        const uint32_t code = TS::LATE_CODES ? zc[a] : codes[s];
        if (code == SLOT_INVALID) return;
        const uint32_t g = code & SLOT_GMASK;
        if (code & SLOT_HALO) {
            if (!(code & SLOT_ESS)) halo[TS::LATE_CODES ? zh[a] : hd[s]] = val;
        } else if (code & SLOT_ESS) {
            y[g] = vess[g];
        } else {
            y[g] = (TOUT)val;
        }
    };
    if (actz) {
        const bool yseam = (zy % K == 0) && zy > 0 && zy < SE - 1;
        float2 z2[Q1];
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            const int qz = Q1 * h + q;
            z2[q] = A2[zx + SE * qz + SA2 * zy];
            if (yseam) z2[q] = __fadd2_rn(SY2[(zy / K - 1) * QT * SE + zx + SE * qz], z2[q]);
        }
        float2 o2[D1];
#pragma unroll
        for (int a = 0; a < D1; ++a) o2[a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < Q1; ++q)
#pragma unroll
            for (int a = 0; a < D1; ++a) o2[a] = __ffma2_rn(Pr.BG[q * D1 + a], z2[q], o2[a]);
#pragma unroll
        for (int a = 0; a < D1; ++a) out[a] = o2[a].x + o2[a].y;
#pragma unroll
        for (int a = 1; a < K; ++a) write_slot(a, out[a]);
        if (h == 0) write_slot(0, out[0]);
        if (h == TT - 1) write_slot(K, out[K]);
        else SZ1[h * SE * SE + L] = out[K];
    }
    bar.sync();
    if (actz && h > 0) write_slot(0, SZ1[(h - 1) * SE * SE + L] + out[0]);
    return true;
}

// Hooks that every thread of a tile runs after its slot codes are requested and before its
// tangent copy and input values; false (uniform across the tile) passes the tile over.
// InputsReady: nothing to wait for.  AfterPriorGrid (the single-instance kernel): wait for the
// grid before this one in the stream (programmatic launch), then pass the tile over if the CG
// flag says that the solve has ended.
struct InputsReady {
    __device__ __forceinline__ bool operator()() const { return true; }
};
struct AfterPriorGrid {
    const int *skip;
    __device__ __forceinline__ bool operator()() const
    {
        grid_dependency_wait();
        return !(skip && *skip);
    }
};

// One tile of the FP32 packed variant on a group of threads (tid: the thread's index in the group,
// bar: the group's barrier) of at least TileShape<D1, TT>::THREADS threads (the extra threads
// take part only in barriers).  smem: the tile's shared region (after the
// mbarrier); mbar: an initialised mbarrier whose phase `parity` this tile's tangent copy
// completes.  Returns false (uniformly) when the tangent copy did not land within the bound;
// the caller then reports and waits for it again.  The slot codes (set-up data) are requested
// first: the input values depend on them, and they are the longest chain of a tile's prologue;
// the tangent copy (waited for only before the x stage) is issued after them.
// TOUT: the output type (TIO unless given); vess: the essential rows' source when TOUT differs
// from TIO (v itself otherwise).
template <int D1, int TT, typename TIO, typename Bar, typename Ready = InputsReady, typename TOUT = TIO>
__device__ __forceinline__ bool tile2_body(const OpParams &P, const BasisPairs &Pr, const float *__restrict__ Tq,
                                           const TIO *__restrict__ v, TOUT *__restrict__ y,
                                           float *__restrict__ halo, int64_t t, unsigned char *smem,
                                           uint64_t *mbar, uint32_t parity, int tid, const Bar &bar,
                                           Ready inputs_ready = Ready{}, const TOUT *vess = nullptr)
{
    using TS = TileShape2<D1, TT>;
    constexpr int NS3 = TS::NS3, NTH = TS::THREADS;
    const int64_t tqs = tq_stride<float>(P);
    const uint32_t tq_bytes = (uint32_t)(tqs * sizeof(float));

    unsigned char *p = smem;
    float *Tb = reinterpret_cast<float *>(p);           p += pad16(tq_bytes);
    uint32_t *codes = reinterpret_cast<uint32_t *>(p);  // shared-memory codes only
    uint32_t *hd = codes + pad16(NS3 * 4) / 4;
    if constexpr (!TS::LATE_CODES) p += TS::CODES_BYTES;
    float2 *A2 = reinterpret_cast<float2 *>(p);         p += pad16((size_t)TS::NA2 * 8);
    float *C1 = reinterpret_cast<float *>(p);           p += pad16((size_t)TS::NC * 4);
    float2 *C2 = reinterpret_cast<float2 *>(p);
    TIO *Vs = reinterpret_cast<TIO *>(C2);              // z stage only; C2 is first written by y
    unsigned char *q = reinterpret_cast<unsigned char *>(Tb);   // seams: after the x stage's reads
    float *SX1 = reinterpret_cast<float *>(q);          q += pad16((size_t)TS::NSX * 4);
    float2 *SX2 = reinterpret_cast<float2 *>(q);        q += pad16((size_t)TS::NSX * 8);
    float2 *SY2 = reinterpret_cast<float2 *>(q);        q += pad16((size_t)TS::NSY * 8);
    float *SZ1 = reinterpret_cast<float *>(q);

    // input gather: slot codes, then (one batch) the input values and, with shared-memory codes,
    // the halo-array positions of halo slots, which reach shared memory after the z stage
    constexpr int NPER = (NS3 + NTH - 1) / NTH;
    uint32_t hr[NPER];
    const bool gth = tid < NTH;
    const uint32_t *sl = P.slot + t * P.Spad;
    const uint32_t *hs = P.hdst + t * P.Spad;
    {
        uint32_t cr[NPER];
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            cr[i] = gth && s < NS3 ? sl[s] : SLOT_INVALID;
        }
        if (!inputs_ready()) return true;
        if (tid == 0) {
            mbar_arrive_expect_tx(mbar, tq_bytes);
            tma_load_1d(Tb, Tq + t * tqs, tq_bytes, mbar);
        }
        TIO vr[NPER];
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            vr[i] = (cr[i] & SLOT_ESS) ? TIO(0) : v[cr[i] & SLOT_GMASK];
            if constexpr (!TS::LATE_CODES) hr[i] = (cr[i] & SLOT_HALO) && !(cr[i] & SLOT_ESS) ? hs[tid + i * NTH] : 0u;
        }
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            if (gth && s < NS3) {
                Vs[s] = vr[i];
                if constexpr (!TS::LATE_CODES) codes[s] = cr[i];
            }
        }
    }
    // makes the gathered block (and, in a new CTA, the mbarrier initialisation) visible to all
    // threads; the tangent block is waited for (bounded) only before the x stage, its first reader
    bar.sync();
    const TOUT *ess;
    if constexpr (std::is_same<TIO, TOUT>::value) ess = vess ? vess : v;
    else ess = vess;
    return tile_stages2<D1, TT, TIO>(
        Pr, Tb, Vs, TS::LATE_CODES ? sl : codes, TS::LATE_CODES ? hs : hd, A2, C1, C2, SX1, SX2, SY2, SZ1, ess, y,
        halo, tid, bar,
        [&]() {
            if constexpr (!TS::LATE_CODES) {
#pragma unroll
                for (int i = 0; i < NPER; ++i) {
                    const int s = tid + i * NTH;
                    if (gth && s < NS3) hd[s] = hr[i];
                }
            }
        },
        [&]() { return !bar.any(!mbar_wait_bounded(mbar, parity)); });
}

// One CTA per tile (FP32 compute; TIO float or double), as k_jv_tile.  Launched
// programmatically after the fix-up of the previous action (outside graph captures): the CTAs
// of its first wave initialise their mbarrier and request their slot codes (set-up data) while
// that fix-up ends, then wait for it before they touch anything a kernel before them wrote.
// TOUT (default TIO): the output type; the CG with FP64 vectors feeds the FP32 rounding of its
// direction (TIO float) and takes an FP64 output, its essential rows copied from vess (the FP64
// direction), so that the result is bit for bit the one of the FP64-input variant on that
// direction.
template <int D1, int TT, typename TIO, typename TOUT = TIO>
__global__ void __launch_bounds__(TileShape<D1, TT>::THREADS)
    k_jv_tile2(const __grid_constant__ OpParams P, const __grid_constant__ BasisPairs Pr,
               const float *__restrict__ Tq, const TIO *__restrict__ v, TOUT *__restrict__ y,
               float *__restrict__ halo, const TOUT *__restrict__ vess)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
    }
    // thread 0 initialises the barrier before it issues the copy; the other threads poll it only
    // after the body's first __syncthreads
    if (!tile2_body<D1, TT, TIO, CtaBar, AfterPriorGrid, TOUT>(P, Pr, Tq, v, y, halo, P.t0 + blockIdx.x, smem + 64,
                                                               mbar, 0u, tid, CtaBar{}, AfterPriorGrid{P.skip},
                                                               vess) && tid == 0) {
        // the tangent block did not land within the bound: report, let the copy finish
        atomicExch(P.err, 3);
        mbar_wait_bounded(mbar, 0);
    }
}

}  // namespace feod
