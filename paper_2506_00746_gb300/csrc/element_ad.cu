// element_ad.cu -- dense element tangent matrices K_e = dr_e/du_e = B^T J_D(u_q) B (Eq. 3), three
// ways, for the comparison of where the AD sits (Table 1's columns):
//   HND: the tangent of the pointwise law written out by hand at each quadrature point;
//   RES: forward AD at the quadrature point (Eq. 2): the law on dual numbers with dim directions;
//   ELM: forward AD at the element level: the element residual r_e = B^T D(B u_e) on dual numbers
//        over the element DOFs (NC directions per pass), so B and B^T sit inside the
//        differentiation.
// HND and RES then form K_e = sum_q G_q^T T_q G_q with G_q the dense 3 x nl reference-gradient
// table at point q.  One CTA loops over elements; the table (the same for every element) is built
// once per CTA in shared memory.  3D, orders 1..3.
#include <algorithm>
#include <cstdio>

#include "element_kernels.cuh"

namespace feod {

enum ElemMethod : int { ELEM_HND = 0, ELEM_RES = 1, ELEM_ELM = 2 };
constexpr int ELEM_THREADS = 256;
constexpr int ELEM_NC = 8;          // dual directions per ELM pass

template <int D1>
struct EShape {
    static constexpr int NL = D1 * D1 * D1;    // element DOFs (= quadrature points)
    static constexpr int NQ = NL;
    static constexpr int ROWS = (NL + ELEM_THREADS / NL - 1) / (ELEM_THREADS / NL);   // rows per thread
};

template <int D1>
__host__ __device__ inline size_t elem_smem_bytes()
{
    using ES = EShape<D1>;
    return (size_t)ES::NQ * 3 * ES::NL * 8      // gradient table gt[q][d][l]
           + (size_t)ES::NL * 8                 // u_e
           + (size_t)ES::NQ * 7 * 8             // M (6), 1/(w detJ) per point
           + (size_t)ES::NQ * 3 * (ELEM_NC + 1) * 8;   // T (6 per point) or the dual flux (ELM)
}

// d tau / d base of kappa(base) = base^a with the limit rule at base == 0 (the derivative term is
// taken as 0 there)
__device__ __forceinline__ double kappa_prime(double base, int law, double a)
{
    switch (law) {
    case LAW_P2: return 0.0;
    case LAW_P3: return base == 0.0 ? 0.0 : 0.5 / sqrt(base);
    case LAW_P4: return 1.0;
    default: return base == 0.0 ? 0.0 : a * pow(base, a - 1.0);
    }
}

template <int D1, int METHOD>
__global__ void __launch_bounds__(ELEM_THREADS)
    k_elem_tangent(const __grid_constant__ OpParams P, const __grid_constant__ BasisT<double> Bs,
                   const double *__restrict__ u, int64_t e0, int64_t count, double *__restrict__ K)
{
    using ES = EShape<D1>;
    constexpr int NL = ES::NL, NQ = ES::NQ, K1 = D1 - 1;
    extern __shared__ __align__(16) unsigned char smem[];
    double *gt = reinterpret_cast<double *>(smem);          // [NQ][3][NL]
    double *ue = gt + NQ * 3 * NL;                           // [NL]
    double *gm = ue + NL;                                    // [NQ][7]
    double *wk = gm + NQ * 7;                                // T [NQ][6] or dual flux [NQ][3][NC+1]
    const int tid = threadIdx.x;
    // reference gradients of every basis function at every point, from the 1D tables
    for (int i = tid; i < NQ * NL; i += ELEM_THREADS) {
        const int q = i / NL, l = i % NL;
        const int qx = q % D1, qy = (q / D1) % D1, qz = q / (D1 * D1);
        const int a = l % D1, b = (l / D1) % D1, c = l / (D1 * D1);
        const double bx = Bs.B[qx * D1 + a], by = Bs.B[qy * D1 + b], bz = Bs.B[qz * D1 + c];
        gt[(q * 3 + 0) * NL + l] = Bs.G[qx * D1 + a] * by * bz;
        gt[(q * 3 + 1) * NL + l] = bx * Bs.G[qy * D1 + b] * bz;
        gt[(q * 3 + 2) * NL + l] = bx * by * Bs.G[qz * D1 + c];
    }
    const int nx = P.n[0], ny = P.n[1], T = P.T;
    const int64_t mx = (int64_t)K1 * nx + 1, my = (int64_t)K1 * ny + 1;
    for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
        const int64_t e = e0 + i;
        const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
        const int64_t t = (ex / T) + (int64_t)P.nt[0] * ((ey / T) + (int64_t)P.nt[1] * (ez / T));
        const int el = (ex % T) + T * ((ey % T) + T * (ez % T));
        const int64_t eint = t * (int64_t)(T * T * T) + el;
        const double *ge = P.geo + eint * (int64_t)(8 * NQ);
        const double kr = P.kr ? P.kr[eint] : 1.0;
        __syncthreads();                                    // previous element done with ue, gm, wk
        for (int l = tid; l < NL; l += ELEM_THREADS) {
            const int a = l % D1, b = (l / D1) % D1, c = l / (D1 * D1);
            ue[l] = u[(K1 * ex + a) + mx * ((K1 * ey + b) + my * (int64_t)(K1 * ez + c))];
        }
        for (int q = tid; q < NQ; q += ELEM_THREADS)
            for (int c = 0; c < 7; ++c) gm[q * 7 + c] = ge[c * NQ + q];
        __syncthreads();
        double *Ke = K + i * (int64_t)NL * NL;
        if constexpr (METHOD != ELEM_ELM) {
            // the point tangent T_q (6 symmetric entries, reference coordinates)
            for (int q = tid; q < NQ; q += ELEM_THREADS) {
                double g[3] = { 0.0, 0.0, 0.0 };
                for (int l = 0; l < NL; ++l)
#pragma unroll
                    for (int d = 0; d < 3; ++d) g[d] += ue[l] * gt[(q * 3 + d) * NL + l];
                double M[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) M[c] = gm[q * 7 + c];
                const double iw = gm[q * 7 + 6];
                double tv[6];
                if constexpr (METHOD == ELEM_HND) {
                    // q = kr kappa(eps^2 + sigma) M g, sigma = g^T M g / (w detJ):
                    // dq/dg = kr (kappa M + 2 kappa' / (w detJ) (M g)(M g)^T)
                    const double m0 = M[0] * g[0] + M[3] * g[1] + M[4] * g[2];
                    const double m1 = M[3] * g[0] + M[1] * g[1] + M[5] * g[2];
                    const double m2 = M[4] * g[0] + M[5] * g[1] + M[2] * g[2];
                    const double base = (g[0] * m0 + g[1] * m1 + g[2] * m2) * iw + P.eps2;
                    const double kap = kr * kappa_of(base, P.law, P.law_a);
                    const double c2 = 2.0 * kr * kappa_prime(base, P.law, P.law_a) * iw;
                    tv[0] = kap * M[0] + c2 * m0 * m0; tv[1] = kap * M[1] + c2 * m1 * m1;
                    tv[2] = kap * M[2] + c2 * m2 * m2; tv[3] = kap * M[3] + c2 * m0 * m1;
                    tv[4] = kap * M[4] + c2 * m0 * m2; tv[5] = kap * M[5] + c2 * m1 * m2;
                } else {
                    Dual<double, 3> gd[3], qd[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        gd[d].v = g[d];
#pragma unroll
                        for (int f = 0; f < 3; ++f) gd[d].d[f] = d == f ? 1.0 : 0.0;
                    }
                    flux3(gd, M, iw, kr, P.law, P.law_a, P.eps2, qd);
                    tv[0] = qd[0].d[0]; tv[1] = qd[1].d[1]; tv[2] = qd[2].d[2];
                    tv[3] = qd[0].d[1]; tv[4] = qd[0].d[2]; tv[5] = qd[1].d[2];
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) wk[q * 6 + c] = tv[c];
            }
            __syncthreads();
            // K_e = sum_q G_q^T T_q G_q: thread (row block rb, column col)
            constexpr int GROUPS = ELEM_THREADS / NL;
            const int col = tid % NL, rb = tid / NL;
            if (rb < GROUPS) {
                double acc[ES::ROWS];
#pragma unroll
                for (int r = 0; r < ES::ROWS; ++r) acc[r] = 0.0;
                for (int q = 0; q < NQ; ++q) {
                    const double *Tq = wk + q * 6;
                    const double gx = gt[(q * 3 + 0) * NL + col], gy = gt[(q * 3 + 1) * NL + col],
                                 gz = gt[(q * 3 + 2) * NL + col];
                    const double w0 = Tq[0] * gx + Tq[3] * gy + Tq[4] * gz;
                    const double w1 = Tq[3] * gx + Tq[1] * gy + Tq[5] * gz;
                    const double w2 = Tq[4] * gx + Tq[5] * gy + Tq[2] * gz;
#pragma unroll
                    for (int r = 0; r < ES::ROWS; ++r) {
                        const int row = rb + GROUPS * r;
                        if (row < NL)
                            acc[r] += gt[(q * 3 + 0) * NL + row] * w0 + gt[(q * 3 + 1) * NL + row] * w1 +
                                      gt[(q * 3 + 2) * NL + row] * w2;
                    }
                }
#pragma unroll
                for (int r = 0; r < ES::ROWS; ++r) {
                    const int row = rb + GROUPS * r;
                    if (row < NL) Ke[(int64_t)row * NL + col] = acc[r];
                }
            }
        } else {
            // element-level forward AD: ELEM_NC element DOF directions per pass
            for (int j0 = 0; j0 < NL; j0 += ELEM_NC) {
                // dual flux at every point: g = sum_l u_l grad phi_l on duals seeded by the pass's DOFs
                for (int q = tid; q < NQ; q += ELEM_THREADS) {
                    Dual<double, ELEM_NC> g[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        g[d].v = 0.0;
#pragma unroll
                        for (int f = 0; f < ELEM_NC; ++f) g[d].d[f] = 0.0;
                    }
                    for (int l = 0; l < NL; ++l) {
                        Dual<double, ELEM_NC> ul;
                        ul.v = ue[l];
#pragma unroll
                        for (int f = 0; f < ELEM_NC; ++f) ul.d[f] = (l == j0 + f) ? 1.0 : 0.0;
#pragma unroll
                        for (int d = 0; d < 3; ++d) g[d] = g[d] + ul * gt[(q * 3 + d) * NL + l];
                    }
                    double M[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) M[c] = gm[q * 7 + c];
                    Dual<double, ELEM_NC> fq[3];
                    flux3(g, M, gm[q * 7 + 6], kr, P.law, P.law_a, P.eps2, fq);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        wk[(q * 3 + d) * (ELEM_NC + 1)] = fq[d].v;
#pragma unroll
                        for (int f = 0; f < ELEM_NC; ++f) wk[(q * 3 + d) * (ELEM_NC + 1) + 1 + f] = fq[d].d[f];
                    }
                }
                __syncthreads();
                // r_l = sum_q grad phi_l(q) . flux(q) on the same duals: column j0 + f of K is d r / d u_j
                for (int l = tid; l < NL; l += ELEM_THREADS) {
                    Dual<double, ELEM_NC> r;
                    r.v = 0.0;
#pragma unroll
                    for (int f = 0; f < ELEM_NC; ++f) r.d[f] = 0.0;
                    for (int q = 0; q < NQ; ++q)
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            Dual<double, ELEM_NC> fq;
                            fq.v = wk[(q * 3 + d) * (ELEM_NC + 1)];
#pragma unroll
                            for (int f = 0; f < ELEM_NC; ++f) fq.d[f] = wk[(q * 3 + d) * (ELEM_NC + 1) + 1 + f];
                            r = r + gt[(q * 3 + d) * NL + l] * fq;
                        }
#pragma unroll
                    for (int f = 0; f < ELEM_NC; ++f)
                        if (j0 + f < NL) Ke[(int64_t)l * NL + j0 + f] = r.d[f];
                }
                __syncthreads();
            }
        }
    }
}

template <int D1, int METHOD>
cudaError_t launch_elem(fe_ctx *c, const double *u, int64_t e0, int64_t count, double *K, cudaStream_t st)
{
    const size_t sm = elem_smem_bytes<D1>();
    cudaError_t e = cudaFuncSetAttribute(k_elem_tangent<D1, METHOD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_elem_tangent<D1, METHOD>, ELEM_THREADS, sm);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(count, (int64_t)std::max(per_sm, 1) * c->num_sms);
    LaunchScope ls(c, METHOD == ELEM_HND ? "elem_tangent_hnd" : METHOD == ELEM_RES ? "elem_tangent_res" : "elem_tangent_elm", st);
    k_elem_tangent<D1, METHOD><<<(unsigned)grid, ELEM_THREADS, sm, st>>>(c->op, c->b64, u, e0, count, K);
    return cudaGetLastError();
}

template <int D1>
cudaError_t launch_elem_m(fe_ctx *c, int method, const double *u, int64_t e0, int64_t count, double *K, cudaStream_t st)
{
    switch (method) {
    case ELEM_HND: return launch_elem<D1, ELEM_HND>(c, u, e0, count, K, st);
    case ELEM_RES: return launch_elem<D1, ELEM_RES>(c, u, e0, count, K, st);
    default: return launch_elem<D1, ELEM_ELM>(c, u, e0, count, K, st);
    }
}

}  // namespace feod

using namespace feod;

extern "C" fe_status fe_element_matrices(fe_ctx *c, const double *u, int method, int64_t e0, int64_t count, double *K,
                                         void *stream)
{
    if (!c) return FE_ERR_ARG;
    if (!u || !K || count < 0 || e0 < 0 || e0 + count > c->ne || method < 0 || method > 2)
        return set_error(c, FE_ERR_ARG, "fe_element_matrices: bad pointer, element range or method");
    if (c->dim != 3 || c->k < 1 || c->k > 3)
        return set_error(c, FE_ERR_UNSUPPORTED, "fe_element_matrices: 3D orders 1..3 only");
    if (count == 0) return FE_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (c->k) {
    case 1: e = launch_elem_m<2>(c, method, u, e0, count, K, st); break;
    case 2: e = launch_elem_m<3>(c, method, u, e0, count, K, st); break;
    default: e = launch_elem_m<4>(c, method, u, e0, count, K, st); break;
    }
    if (e != cudaSuccess) return set_error(c, FE_ERR_CUDA, cudaGetErrorString(e));
    return FE_OK;
}
