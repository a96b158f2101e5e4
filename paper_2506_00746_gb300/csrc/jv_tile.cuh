// jv_tile.cuh -- partially assembled Jacobian action with tile-level sum factorisation (3D).
//
// y = P^T G^T B^T (T_q . B G P v) for one tile of TT^3 elements per CTA.  On a structured tile
// the element restriction G and the 1D basis operators compose into block-sparse 1D operators
//     Bt[Q1 e + q][K e + a] = B^[q][a],   Gt[Q1 e + q][K e + a] = G^[q][a]   (e < TT, a <= K),
// acting between the tile's SE = K TT + 1 DOF slots and QT = Q1 TT quadrature points per
// direction.  Sum factorisation over the tile therefore applies B G to the tile's DOF block
// directly (no per-element copies) and the transposed contractions apply G^T B^T: the DOF shared
// by neighbouring elements of the tile receives both elements' terms inside the contraction, in
// ascending element order, so the in-tile G^T is exact, deterministic and free.  Slots on the
// tile's upper faces that belong to a neighbouring tile go to the halo buffer as before.
//
// Per CTA: one bulk copy (TMA, mbarrier-completed, bounded wait) brings the tile's stored
// tangent block into shared memory while the threads gather the DOF block; then five line
// stages (z, y, x+D+x^T, y^T, z^T), each thread owning one line of the current direction, with
// shared-memory layouts chosen so that lanes of a warp touch consecutive or odd-strided words.
#pragma once

namespace feod {

__host__ __device__ inline size_t pad16(size_t b) { return (b + 15) & ~(size_t)15; }

template <int D1, int TT>
struct TileShape {
    static constexpr int K = D1 - 1;
    static constexpr int SE = K * TT + 1;          // DOF slots per tile edge
    static constexpr int QT = D1 * TT;             // quadrature points per tile edge
    static constexpr int NS3 = SE * SE * SE;
    static constexpr int NQT = QT * QT * QT;
    static constexpr int NA = SE * QT * SE;        // one z- or y-stage array
    static constexpr int NC = QT * QT * SE;        // one x-stage array
    static constexpr int THREADS = ((QT * QT + 31) / 32) * 32;
};

template <int D1, int TT, typename TC>
__host__ __device__ inline size_t tile_smem_bytes(int64_t tqs)
{
    using TS = TileShape<D1, TT>;
    return 16 + pad16((size_t)tqs * sizeof(TC)) + pad16(TS::NS3 * sizeof(TC)) + pad16(TS::NS3 * 4) +
           pad16(2 * (size_t)TS::NA * sizeof(TC)) + 3 * (size_t)TS::NC * sizeof(TC);
}

// n consecutive shared-memory values into registers; 16-byte vector loads when n % 4 == 0 (FP32)
// or n % 2 == 0 (FP64) -- the caller guarantees the alignment in those cases.
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
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const double2 w = *reinterpret_cast<const double2 *>(p + i);
            r[i] = w.x; r[i + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = p[i];
    }
}

template <int D1, int TT, typename TC, typename TIO>
__global__ void __launch_bounds__(TileShape<D1, TT>::THREADS)
    k_jv_tile(const __grid_constant__ OpParams P, const __grid_constant__ BasisT<TC> Bs, const TC *__restrict__ Tq,
              const TIO *__restrict__ v, TIO *__restrict__ y, TC *__restrict__ halo)
{
    using TS = TileShape<D1, TT>;
    constexpr int K = TS::K, Q1 = D1, SE = TS::SE, QT = TS::QT, NS3 = TS::NS3, NQT = TS::NQT;
    constexpr int NA = TS::NA, NC = TS::NC, NTH = TS::THREADS;
    if (P.skip && *P.skip) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const int64_t t = blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t tqs = tq_stride<TC>(P);
    const uint32_t tq_bytes = (uint32_t)(tqs * sizeof(TC));

    unsigned char *p = smem;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(p);    p += 16;
    TC *Tb = reinterpret_cast<TC *>(p);                 p += pad16(tq_bytes);            // [c][qz][qy][qx]
    TC *Vs = reinterpret_cast<TC *>(p);                 p += pad16(NS3 * sizeof(TC));    // [sz][sy][sx]
    uint32_t *codes = reinterpret_cast<uint32_t *>(p);  p += pad16(NS3 * 4);
    TC *AE = reinterpret_cast<TC *>(p);                 p += pad16(2 * NA * sizeof(TC)); // [arr][sy][qz][sx]
    TC *Cb = reinterpret_cast<TC *>(p);                                                   // [arr][qz][qy][sx]

    // the tile's tangent block: one bulk copy, in flight while the DOF block is gathered
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(mbar, tq_bytes);
        tma_load_1d(Tb, Tq + t * tqs, tq_bytes, mbar);
    }
    // G and P: slot codes, then all of this thread's input values at once
    {
        constexpr int NPER = (NS3 + NTH - 1) / NTH;
        const uint32_t *sl = P.slot + t * P.Spad;
        uint32_t cr[NPER];
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            cr[i] = s < NS3 ? sl[s] : SLOT_INVALID;
        }
        TC vr[NPER];
#pragma unroll
        for (int i = 0; i < NPER; ++i) vr[i] = (cr[i] & SLOT_ESS) ? TC(0) : (TC)v[cr[i] & SLOT_GMASK];
#pragma unroll
        for (int i = 0; i < NPER; ++i) {
            const int s = tid + i * NTH;
            if (s < NS3) { codes[s] = cr[i]; Vs[s] = vr[i]; }
        }
    }
    __syncthreads();

    // z: line (sx, sy) of SE slots -> QT points, B^ and G^
    if (tid < SE * SE) {
        const int sx = tid % SE, sy = tid / SE;
        TC in[SE];
#pragma unroll
        for (int sz = 0; sz < SE; ++sz) in[sz] = Vs[(sz * SE + sy) * SE + sx];
#pragma unroll
        for (int e = 0; e < TT; ++e)
#pragma unroll
            for (int q = 0; q < Q1; ++q) {
                TC a0 = TC(0), a1 = TC(0);
#pragma unroll
                for (int a = 0; a < D1; ++a) {
                    a0 += Bs.B[q * D1 + a] * in[K * e + a];
                    a1 += Bs.G[q * D1 + a] * in[K * e + a];
                }
                const int o = (sy * QT + Q1 * e + q) * SE + sx;
                AE[o] = a0;
                AE[NA + o] = a1;
            }
    }
    __syncthreads();
    // y: line (sx, qz)
    if (tid < SE * QT) {
        const int sx = tid % SE, qz = tid / SE;
        TC a0[SE], a1[SE];
#pragma unroll
        for (int sy = 0; sy < SE; ++sy) {
            a0[sy] = AE[(sy * QT + qz) * SE + sx];
            a1[sy] = AE[NA + (sy * QT + qz) * SE + sx];
        }
#pragma unroll
        for (int e = 0; e < TT; ++e)
#pragma unroll
            for (int q = 0; q < Q1; ++q) {
                TC c00 = TC(0), c01 = TC(0), c10 = TC(0);
#pragma unroll
                for (int a = 0; a < D1; ++a) {
                    c00 += Bs.B[q * D1 + a] * a0[K * e + a];
                    c01 += Bs.G[q * D1 + a] * a0[K * e + a];
                    c10 += Bs.B[q * D1 + a] * a1[K * e + a];
                }
                const int o = (qz * QT + Q1 * e + q) * SE + sx;
                Cb[o] = c00;
                Cb[NC + o] = c01;
                Cb[2 * NC + o] = c10;
            }
    }
    // the tangent block must have landed (bounded wait; uniform decision, doubles as the barrier)
    const bool bad = !mbar_wait_bounded(mbar, 0);
    if (__syncthreads_or(bad)) {
        if (tid == 0) {
            atomicExch(P.err, 3);
            mbar_wait_bounded(mbar, 0);
        }
        return;
    }
    // x: line (qy, qz); gradient, D (stored tangent), and the x transpose, element by element
    if (tid < QT * QT) {
        const int qy = tid % QT, qz = tid / QT;
        const int o = (qz * QT + qy) * SE;
        TC c00[SE], c01[SE], c10[SE], d00[SE], d01[SE], d10[SE];
#pragma unroll
        for (int sx = 0; sx < SE; ++sx) {
            c00[sx] = Cb[o + sx]; c01[sx] = Cb[NC + o + sx]; c10[sx] = Cb[2 * NC + o + sx];
            d00[sx] = TC(0); d01[sx] = TC(0); d10[sx] = TC(0);
        }
        const TC *Tl = Tb + (qz * QT + qy) * QT;
#pragma unroll
        for (int e = 0; e < TT; ++e) {
            TC txx[Q1], tyy[Q1], tzz[Q1], txy[Q1], txz[Q1], tyz[Q1];
            lds_run<Q1, TC>(Tl + Q1 * e, txx);
            lds_run<Q1, TC>(Tl + NQT + Q1 * e, tyy);
            lds_run<Q1, TC>(Tl + 2 * NQT + Q1 * e, tzz);
            lds_run<Q1, TC>(Tl + 3 * NQT + Q1 * e, txy);
            lds_run<Q1, TC>(Tl + 4 * NQT + Q1 * e, txz);
            lds_run<Q1, TC>(Tl + 5 * NQT + Q1 * e, tyz);
#pragma unroll
            for (int q = 0; q < Q1; ++q) {
                TC gx = TC(0), gy = TC(0), gz = TC(0);
#pragma unroll
                for (int a = 0; a < D1; ++a) {
                    gx += Bs.G[q * D1 + a] * c00[K * e + a];
                    gy += Bs.B[q * D1 + a] * c01[K * e + a];
                    gz += Bs.B[q * D1 + a] * c10[K * e + a];
                }
                const TC fx = txx[q] * gx + txy[q] * gy + txz[q] * gz;
                const TC fy = txy[q] * gx + tyy[q] * gy + tyz[q] * gz;
                const TC fz = txz[q] * gx + tyz[q] * gy + tzz[q] * gz;
#pragma unroll
                for (int a = 0; a < D1; ++a) {
                    d00[K * e + a] += Bs.G[q * D1 + a] * fx;
                    d01[K * e + a] += Bs.B[q * D1 + a] * fy;
                    d10[K * e + a] += Bs.B[q * D1 + a] * fz;
                }
            }
        }
#pragma unroll
        for (int sx = 0; sx < SE; ++sx) {
            Cb[o + sx] = d00[sx]; Cb[NC + o + sx] = d01[sx]; Cb[2 * NC + o + sx] = d10[sx];
        }
    }
    __syncthreads();
    // y transpose: line (sx, qz)
    if (tid < SE * QT) {
        const int sx = tid % SE, qz = tid / SE;
        TC e00[QT], e01[QT], e10[QT], E0[SE], E1[SE];
#pragma unroll
        for (int qy = 0; qy < QT; ++qy) {
            const int o = (qz * QT + qy) * SE + sx;
            e00[qy] = Cb[o]; e01[qy] = Cb[NC + o]; e10[qy] = Cb[2 * NC + o];
        }
#pragma unroll
        for (int s = 0; s < SE; ++s) { E0[s] = TC(0); E1[s] = TC(0); }
#pragma unroll
        for (int e = 0; e < TT; ++e)
#pragma unroll
            for (int q = 0; q < Q1; ++q)
#pragma unroll
                for (int a = 0; a < D1; ++a) {
                    E0[K * e + a] += Bs.B[q * D1 + a] * e00[Q1 * e + q] + Bs.G[q * D1 + a] * e01[Q1 * e + q];
                    E1[K * e + a] += Bs.B[q * D1 + a] * e10[Q1 * e + q];
                }
#pragma unroll
        for (int sy = 0; sy < SE; ++sy) {
            const int o = (sy * QT + qz) * SE + sx;
            AE[o] = E0[sy];
            AE[NA + o] = E1[sy];
        }
    }
    __syncthreads();
    // z transpose: line (sx, sy); then P^T and the writes (halo slots to the fix-up buffer)
    if (tid < SE * SE) {
        const int sx = tid % SE, sy = tid / SE;
        TC z0[QT], z1[QT], out[SE];
#pragma unroll
        for (int qz = 0; qz < QT; ++qz) {
            z0[qz] = AE[(sy * QT + qz) * SE + sx];
            z1[qz] = AE[NA + (sy * QT + qz) * SE + sx];
        }
#pragma unroll
        for (int s = 0; s < SE; ++s) out[s] = TC(0);
#pragma unroll
        for (int e = 0; e < TT; ++e)
#pragma unroll
            for (int q = 0; q < Q1; ++q)
#pragma unroll
                for (int a = 0; a < D1; ++a)
                    out[K * e + a] += Bs.B[q * D1 + a] * z0[Q1 * e + q] + Bs.G[q * D1 + a] * z1[Q1 * e + q];
#pragma unroll
        for (int sz = 0; sz < SE; ++sz) {
            const int s = (sz * SE + sy) * SE + sx;
            const uint32_t code = codes[s];
            if (code == SLOT_INVALID) continue;
            const uint32_t g = code & SLOT_GMASK;
            if (code & SLOT_HALO) {
                if (!(code & SLOT_ESS)) halo[t * P.Spad + s] = out[sz];
            } else if (code & SLOT_ESS) {
                y[g] = v[g];
            } else {
                y[g] = (TIO)out[sz];
            }
        }
    }
}

}  // namespace feod
