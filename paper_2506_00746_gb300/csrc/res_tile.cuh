// res_tile.cuh -- residual R(u) and quadrature-point tangent J_D with tile-level collocated sum
// factorisation (3D, FP64).
//
// The stages of the collocated tile kernel (jv_tile.cuh) with the pointwise operator D in place
// of the stored tangent (Eq. 1, Eq. 2).  Per tile of TT^3 elements, one CTA:
//   prologue  the tile's DOF block of u through the slot codes (u keeps its boundary values);
//   z, y, x1  interpolation to the quadrature points (B along z, y, x);
//   x2        the reference gradient g (collocation derivative), the point's geometric factors
//             (M = w detJ J^-1 J^-T, 1/(w detJ), w detJ f) from global memory, and the flux
//             q = kappa_rho kappa(eps^2 + |grad u|^2) M g -- on reals (residual only), or on dual
//             numbers seeded with the unit directions of g, whose derivative part is the tangent
//             dq/dg (forward-mode AD at the quadrature point, Eq. 2), stored in the tile layout of
//             the partially assembled J v (FP64 and/or FP32);
//   x3 .. zT  (residual only) W = Dc^T q - w detJ f at the points, then B^T along x, y, z, the
//             seams and the writes: essential rows R = 0, halo slots to the cross-tile buffer,
//             the tile's own DOFs to r (the fix-up kernel adds the halo partial sums).
// A ragged last tile needs no special case: its padded elements have zero geometric factors, so
// their flux, load term and tangent are exact zeros, and their slots have invalid codes.
#pragma once

namespace feod {

// Writes of one tile's residual: P^T (essential rows R = 0; a halo slot of an essential DOF is
// dropped, its owner writes the 0), the halo partial sums, the tile's own DOFs.
struct ResWriter {
    const uint32_t *codes, *hd;
    double *r;
    double *halo;
    __device__ void operator()(int s, double val) const
    {
        const uint32_t code = codes[s];
        if (code == SLOT_INVALID) return;
        if (code & SLOT_HALO) {
            if (!(code & SLOT_ESS)) halo[hd[s]] = val;
        } else {
            r[code & SLOT_GMASK] = (code & SLOT_ESS) ? 0.0 : val;
        }
    }
};

// Shared memory of k_res_tile: the collocated tile layout with no tangent block (its region holds
// only the seam planes).
template <int D1, int TT>
__host__ __device__ inline size_t res_tile_smem_bytes()
{
    return TileLayout<D1, TT, double, double>(0).total;
}

// x2 of the residual: gradient, geometric factors and flux at this thread's Q1 points (the
// x-line segment h of point column (qy, qz)); fx, sv: the x-flux and the load term -w detJ f at
// those points (registers, read back by x3 on the same thread); FY, FZ: the other flux
// components.  TAN: the flux on dual numbers, its derivative stored to T64 / T32 (non-null).
template <int D1, int TT, bool TAN>
__device__ __forceinline__ void res_x2(const OpParams &P, const BasisT<double> &Bs, int64_t t, const double *U,
                                       double (&fx)[D1], double (&sv)[D1], double *FY, double *FZ,
                                       double *__restrict__ T64, float *__restrict__ T32, int tid)
{
    using S = Colloc<D1, TT>;
    constexpr int Q1 = D1, QT = S::QT, NQT = S::NQT;
    constexpr int NQ = D1 * D1 * D1, NE = TT * TT * TT;
    int L, h;
    if (!S::template line<QT * QT>(tid, L, h)) return;
    const int qz = L % QT, qy = L / QT;
    const int ey = qy / Q1, yl = qy % Q1, ez = qz / Q1, zl = qz % Q1;
    const int y0 = Q1 * ey, z0 = Q1 * ez;

    // the element (x column h of the tile) and its point (0, yl, zl): the thread's Q1 points are
    // consecutive in the element's point order q = qx + D1 (qy + D1 qz)
    const int64_t eint = t * NE + h + TT * (ey + TT * ez);
    const double *__restrict__ ge = P.geo + eint * (int64_t)(8 * NQ) + D1 * (yl + D1 * zl);
    const double kr = P.kr ? __ldg(P.kr + eint) : 1.0;

    double u[Q1];
#pragma unroll
    for (int j = 0; j < Q1; ++j) u[j] = U[S::pidx(Q1 * h + j, qy, qz)];
    double gxs[Q1], gys[Q1], gzs[Q1];
#pragma unroll
    for (int q = 0; q < Q1; ++q) { gxs[q] = 0.0; gys[q] = 0.0; gzs[q] = 0.0; }
#pragma unroll
    for (int j = 0; j < Q1; ++j)
#pragma unroll
        for (int q = 0; q < Q1; ++q) {
            const int qx = Q1 * h + q;
            gxs[q] += Bs.Dc[q * Q1 + j] * u[j];
            gys[q] += Bs.Dc[yl * Q1 + j] * U[S::pidx(qx, y0 + j, qz)];
            gzs[q] += Bs.Dc[zl * Q1 + j] * U[S::pidx(qx, qy, z0 + j)];
        }

    // tile-layout offset of the thread's first point in each tangent component block
    const int to = Q1 * (qz + QT * (qy + QT * h));
#pragma unroll
    for (int q = 0; q < Q1; ++q) {
        double M[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) M[c] = __ldg(ge + c * NQ + q);
        const double iw = __ldg(ge + 6 * NQ + q);
        sv[q] = -__ldg(ge + 7 * NQ + q);
        double f[3];
        if constexpr (TAN) {
            Dual<double, 3> gd[3], qd[3];
            const double gq[3] = { gxs[q], gys[q], gzs[q] };
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                gd[d].v = gq[d];
#pragma unroll
                for (int e = 0; e < 3; ++e) gd[d].d[e] = (d == e) ? 1.0 : 0.0;
            }
            flux3(gd, M, iw, kr, P.law, P.law_a, P.eps2, qd);
            // upper triangle of dq/dg: xx yy zz xy xz yz
            const double tv[6] = { qd[0].d[0], qd[1].d[1], qd[2].d[2], qd[0].d[1], qd[0].d[2], qd[1].d[2] };
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                if (T64) T64[t * P.tqs64 + c * NQT + to + q] = tv[c];
                if (T32) T32[t * P.tqs32 + c * NQT + to + q] = (float)tv[c];
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) f[d] = qd[d].v;
        } else {
            const double gq[3] = { gxs[q], gys[q], gzs[q] };
            flux3(gq, M, iw, kr, P.law, P.law_a, P.eps2, f);
        }
        fx[q] = f[0];
        FY[S::pidx(Q1 * h + q, qy, qz)] = f[1];
        FZ[S::pidx(Q1 * h + q, qy, qz)] = f[2];
    }
}

// One CTA per tile.  RES: write R(u) (halo partial sums for the fix-up); TAN: store the tangent.
template <int D1, int TT, bool RES, bool TAN>
__global__ void __launch_bounds__(TileShape<D1, TT>::CTHREADS, tile_min_blocks<TileShape<D1, TT>::CTHREADS>())
    k_res_tile(const __grid_constant__ OpParams P, const __grid_constant__ BasisT<double> Bs,
               const double *__restrict__ u, double *__restrict__ r, double *__restrict__ halo,
               double *__restrict__ T64, float *__restrict__ T32)
{
    using TS = TileShape<D1, TT>;
    using S = Colloc<D1, TT>;
    constexpr int NS3 = TS::NS3, NSX = TS::NSX, NSY = TS::NSY, NTH = TS::CTHREADS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t t = P.t0 + blockIdx.x;
    const int tid = threadIdx.x;

    const TileLayout<D1, TT, double, double> lay(0);
    double *SX = reinterpret_cast<double *>(smem + lay.tb);    // x3 .. seam
    double *SY = SX + NSX;
    double *SZ = SY + NSY;
    uint32_t *codes = reinterpret_cast<uint32_t *>(smem + lay.codes);
    uint32_t *hd = reinterpret_cast<uint32_t *>(smem + lay.hd);
    double *A = reinterpret_cast<double *>(smem + lay.a);
    double *U = A;                                               // x1 .. x2
    double *C = reinterpret_cast<double *>(smem + lay.c);
    double *Vs = C;                                              // prologue .. z
    double *FY = reinterpret_cast<double *>(smem + lay.fy);
    double *FZ = reinterpret_cast<double *>(smem + lay.fz);

    {
        constexpr int NPER = (NS3 + NTH - 1) / NTH;
        const uint32_t *sl = P.slot + t * P.Spad;
        const uint32_t *hs = P.hdst + t * P.Spad;
        uint32_t cr[NPER], hr[NPER];
        double vr[NPER];
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            cr[i] = s < NS3 ? sl[s] : SLOT_INVALID;
        }
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            vr[i] = cr[i] == SLOT_INVALID ? 0.0 : u[cr[i] & SLOT_GMASK];
            hr[i] = RES && (cr[i] != SLOT_INVALID) && (cr[i] & SLOT_HALO) && !(cr[i] & SLOT_ESS) ? hs[tid + i * NTH] : 0u;
        }
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            if (s < NS3) {
                Vs[s] = vr[i];
                if constexpr (RES) { codes[s] = cr[i]; hd[s] = hr[i]; }
            }
        }
    }
    __syncthreads();
    S::z(Bs, Vs, A, tid);
    __syncthreads();
    S::y(Bs, A, C, tid);
    __syncthreads();
    S::x1(Bs, C, U, tid);
    __syncthreads();
    double fx[D1], sv[D1];
    res_x2<D1, TT, TAN>(P, Bs, t, U, fx, sv, FY, FZ, T64, T32, tid);
    if constexpr (RES) {
        __syncthreads();
        // the transposed stages on work units (seams folded in first), except at order 5, where
        // their registers cost this kernel more than the idle lanes they save (2.46 -> 2.63 ms
        // at 8M DOFs; orders 1-4 and 6 gained 1-6 %)
        constexpr bool TU = D1 != 6;
        S::template x3s<double, true>(Bs, fx, sv, FY, FZ, C, SX, tid);
        __syncthreads();
        if constexpr (TU) {
            S::foldx(C, SX, tid);
            __syncthreads();
        }
        S::template yT<double, TU>(Bs, C, SX, A, SY, tid);
        __syncthreads();
        if constexpr (TU) {
            S::foldy(A, SY, tid);
            __syncthreads();
        }
        const ResWriter write{ codes, hd, r, halo };
        double out0 = 0.0;
        S::template zT<double, ResWriter, TU>(Bs, A, SY, SZ, write, out0, tid);
        __syncthreads();
        S::template seam<double, ResWriter, TU>(SZ, write, out0, tid);
    }
}

}  // namespace feod
