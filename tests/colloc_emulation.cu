// Host run of the collocated tile stages (Colloc<D1, TT> of the generic FP64 / double-float tile
// kernel) against a per-element tensor-product Jacobian action on the same tile.  Each stage is a
// host-callable function of the thread index; a loop over the thread indices runs it between the
// same barriers as the kernel, once with the threads of each stage in ascending and once in
// descending order, in the kernel's shared-memory aliasing (TileLayout).  Random slot values and a
// random symmetric tangent per point; every work array sits between guard regions (an access outside reads a huge sentinel or overwrites
// one) and starts as NaN (a read of an unwritten entry shows in the result).  Checks, per tile
// shape: agreement with the reference to 1e-13 of its largest entry, every slot written exactly
// once, no guard touched, every output finite.  Also: the collocation derivative table is exact on
// polynomials of degree < Q1.  Exit status 0 when everything passes.
#include "element_kernels.cuh"
#include <cstdio>
#include <cmath>
#include <random>
namespace feod {
void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &w);
void gll_nodes(int k, std::vector<double> &x);
void lagrange_tables(const std::vector<double> &nodes, const std::vector<double> &pts, std::vector<double> &val,
                     std::vector<double> &der);
}
using namespace feod;

template <int D1, int TT>
double run(unsigned seed, bool reverse)
{
    using TS = TileShape<D1, TT>;
    using S = Colloc<D1, TT>;
    using L = TileLayout<D1, TT, double, double>;
    constexpr int K = TS::K, Q1 = D1, SE = TS::SE, QT = TS::QT, NQT = TS::NQT, NS3 = TS::NS3;
    BasisT<double> Bs{};
    std::vector<double> gx, gw, nodes, val, der, cval, cder;
    gauss_legendre(Q1, gx, gw); gll_nodes(K, nodes);
    std::vector<double> xq(Q1), xn(D1);
    for (int q = 0; q < Q1; ++q) xq[q] = 0.5 * (gx[q] + 1.0);
    for (int a = 0; a < D1; ++a) xn[a] = 0.5 * (nodes[a] + 1.0);
    lagrange_tables(xn, xq, val, der);
    lagrange_tables(xq, xq, cval, cder);
    for (int i = 0; i < Q1 * D1; ++i) { Bs.B[i] = val[i]; Bs.G[i] = der[i]; }
    for (int i = 0; i < Q1 * Q1; ++i) Bs.Dc[i] = cder[i];
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U01(-1.0, 1.0);
    std::vector<double> Vs(NS3), Tb(6 * NQT);
    for (auto &x : Vs) x = U01(rng);
    for (auto &x : Tb) x = U01(rng);
    // emulated shared memory (poisoned with NaN so that an unwritten read shows)
    const double nan = std::nan("");
    // every array sits between guard regions of 4096 sentinels; any access outside reads a
    // sentinel (huge, shows in the result) or overwrites one (checked below)
    constexpr int GRD = 4096;
    const double SENT = 1e300;
    std::vector<std::vector<double>> store;
    auto arr = [&](int n, double fill) {
        store.emplace_back(std::vector<double>(n + 2 * GRD, SENT));
        for (int i = 0; i < n; ++i) store.back()[GRD + i] = fill;
        return store.size() - 1;
    };
    // the kernel's aliasing: U inside A, the gathered block inside C, the seam planes inside the
    // tangent block (region sizes as TileLayout allocates them)
    const int nTb = (int)(std::max(L(6 * NQT).codes - L(6 * NQT).tb, L::SEAM_ELEMS * sizeof(double)) / sizeof(double));
    const size_t iA = arr((int)(L::A_BYTES / sizeof(double)), nan), iC = arr((int)(L::C_BYTES / sizeof(double)), nan),
                 iTb = arr(nTb, nan), iFY = arr(NQT, nan), iFZ = arr(NQT, nan);
    auto P_ = [&](size_t i) { return store[i].data() + GRD; };
    double *A = P_(iA), *C = P_(iC), *Tbs = P_(iTb), *FY = P_(iFY), *FZ = P_(iFZ);
    double *Uq = A, *Vss = C;
    double *SX = Tbs, *SY = SX + TS::NSX, *SZ = SY + TS::NSY;
    for (int s = 0; s < NS3; ++s) Vss[s] = Vs[s];
    for (int i = 0; i < 6 * NQT; ++i) Tbs[i] = Tb[i];
    std::vector<double> fxs((size_t)TS::CTHREADS * Q1, nan);     // each thread's registers
    std::vector<uint32_t> codes(NS3), hd(NS3, 0);
    for (int s = 0; s < NS3; ++s) codes[s] = (uint32_t)s;
    std::vector<double> v(NS3, 0.0), y(NS3, nan), halo(1, 0.0), out0(TS::CTHREADS, 0.0);
    std::vector<int> writes(NS3, 0);
    struct CountingWriter {
        SlotWriter<double, double> w; int *cnt;
        void operator()(int s, double val) const { cnt[s]++; w(s, val); }
    } write{ SlotWriter<double, double>{ codes.data(), hd.data(), v.data(), y.data(), halo.data() }, writes.data() };
    const int NT = TS::CTHREADS;
    // threads of a stage in ascending or descending order: a write of one thread that another
    // thread of the same stage still reads shows in one of the two orders
    auto each = [&](auto &&stage) {
        for (int i = 0; i < NT; ++i) stage(reverse ? NT - 1 - i : i);
    };
    each([&](int t) { S::z(Bs, Vss, A, t); });
    each([&](int t) { S::y(Bs, A, C, t); });
    each([&](int t) { S::x1(Bs, C, Uq, t); });
    each([&](int t) { S::x2(Bs, Tbs, Uq, fxs.data() + (size_t)t * Q1, FY, FZ, t); });
    each([&](int t) { S::x3(Bs, fxs.data() + (size_t)t * Q1, FY, FZ, C, SX, t); });
    if constexpr (S::template UNITS<double>) each([&](int t) { S::foldx(C, SX, t); });
    each([&](int t) { S::yT(Bs, C, SX, A, SY, t); });
    if constexpr (S::template UNITS<double>) each([&](int t) { S::foldy(A, SY, t); });
    each([&](int t) { S::zT(Bs, A, SY, SZ, write, out0[t], t); });
    each([&](int t) { S::seam(SZ, write, out0[t], t); });
    // reference: per element, full tensor products
    std::vector<double> yr(NS3, 0.0);
    for (int ez = 0; ez < TT; ++ez) for (int ey = 0; ey < TT; ++ey) for (int ex = 0; ex < TT; ++ex)
    for (int qz = 0; qz < Q1; ++qz) for (int qy = 0; qy < Q1; ++qy) for (int qx = 0; qx < Q1; ++qx) {
        double g[3] = { 0, 0, 0 };
        for (int c = 0; c < D1; ++c) for (int b = 0; b < D1; ++b) for (int a = 0; a < D1; ++a) {
            const int s = ((ez * K + c) * SE + ey * K + b) * SE + ex * K + a;
            const double Bx = Bs.B[qx * D1 + a], By = Bs.B[qy * D1 + b], Bz = Bs.B[qz * D1 + c];
            const double Gx = Bs.G[qx * D1 + a], Gy = Bs.G[qy * D1 + b], Gz = Bs.G[qz * D1 + c];
            g[0] += Gx * By * Bz * Vs[s]; g[1] += Bx * Gy * Bz * Vs[s]; g[2] += Bx * By * Gz * Vs[s];
        }
        const int ti = ((ex * QT + ey * Q1 + qy) * QT + ez * Q1 + qz) * Q1 + qx;
        const double txx = Tb[ti], tyy = Tb[NQT + ti], tzz = Tb[2 * NQT + ti];
        const double txy = Tb[3 * NQT + ti], txz = Tb[4 * NQT + ti], tyz = Tb[5 * NQT + ti];
        const double f[3] = { txx * g[0] + txy * g[1] + txz * g[2], txy * g[0] + tyy * g[1] + tyz * g[2],
                              txz * g[0] + tyz * g[1] + tzz * g[2] };
        for (int c = 0; c < D1; ++c) for (int b = 0; b < D1; ++b) for (int a = 0; a < D1; ++a) {
            const int s = ((ez * K + c) * SE + ey * K + b) * SE + ex * K + a;
            const double Bx = Bs.B[qx * D1 + a], By = Bs.B[qy * D1 + b], Bz = Bs.B[qz * D1 + c];
            const double Gx = Bs.G[qx * D1 + a], Gy = Bs.G[qy * D1 + b], Gz = Bs.G[qz * D1 + c];
            yr[s] += Gx * By * Bz * f[0] + Bx * Gy * Bz * f[1] + Bx * By * Gz * f[2];
        }
    }
    double err = 0.0, nrm = 0.0;
    int bad_writes = 0, guards = 0, nonfinite = 0;
    for (auto &a : store) {
        for (int i = 0; i < GRD; ++i) guards += (a[i] != SENT) + (a[a.size() - 1 - i] != SENT);
    }
    for (int s = 0; s < NS3; ++s) nonfinite += !std::isfinite(y[s]) || std::fabs(y[s]) > 1e100;
    for (int s = 0; s < NS3; ++s) {
        err = std::max(err, std::fabs(y[s] - yr[s]));
        nrm = std::max(nrm, std::fabs(yr[s]));
        if (writes[s] != 1) ++bad_writes;
    }
    printf("D1=%d TT=%d threads=%d %s  max|y-yref|/max|yref| = %.3e  slots written != once: %d  guards hit: %d  "
           "non-finite: %d\n", D1, TT, NT, reverse ? "descending" : "ascending ", err / nrm, bad_writes, guards,
           nonfinite);
    return (bad_writes == 0 && guards == 0 && nonfinite == 0 && err / nrm < 1e-13) ? 0.0 : 1.0;
}

// The FP32 tile variants that load the last stage's slot codes from global memory: those whose
// shared-memory-limited CTAs per SM rise without the codes.  Single-instance kernel: orders 3-6
// (9 -> 10, 4 -> 5, 2 -> 3, 12 -> 14 CTAs per SM), not orders 1-2.  Batch variants: the order-4
// one-element tile (28 -> 32), not the other small ones (already at 16 or 32).
static_assert(!TileShape2<2, 4>::LATE_CODES && !TileShape2<3, 3>::LATE_CODES, "orders 1-2 keep shared-memory codes");
static_assert(TileShape2<4, 2>::LATE_CODES && TileShape2<5, 2>::LATE_CODES && TileShape2<6, 2>::LATE_CODES &&
                  TileShape2<7, 1>::LATE_CODES,
              "orders 3-6 load late codes");
static_assert(!TileShape2<2, 2>::LATE_CODES && !TileShape2<3, 2>::LATE_CODES && !TileShape2<3, 1>::LATE_CODES &&
                  !TileShape2<4, 1>::LATE_CODES && TileShape2<5, 1>::LATE_CODES,
              "batch variants: only the order-4 one-element tile loads late codes");

// The collocation derivative on Q1 Gauss points is exact on polynomials of degree < Q1: for
// p(x) = x^m, sum_j Dc[q][j] p(x_j) = m x_q^(m-1) at every Gauss point (x on [0, 1]).
double check_dc(int q1)
{
    std::vector<double> gx, gw, xq(q1), cval, cder;
    gauss_legendre(q1, gx, gw);
    for (int q = 0; q < q1; ++q) xq[q] = 0.5 * (gx[q] + 1.0);
    lagrange_tables(xq, xq, cval, cder);
    double worst = 0.0;
    for (int m = 0; m < q1; ++m)
        for (int q = 0; q < q1; ++q) {
            double d = 0.0;
            for (int j = 0; j < q1; ++j) d += cder[q * q1 + j] * std::pow(xq[j], m);
            const double exact = m == 0 ? 0.0 : m * std::pow(xq[q], m - 1);
            worst = std::max(worst, std::fabs(d - exact));
        }
    printf("Q1=%d collocation derivative: max error on x^m, m < Q1: %.3e\n", q1, worst);
    return worst < 1e-12 ? 0.0 : 1.0;
}

int main()
{
    double bad = 0;
    for (int q1 = 2; q1 <= 7; ++q1) bad += check_dc(q1);
    for (bool rev : { false, true }) {
        bad += run<2, 4>(1, rev); bad += run<3, 3>(2, rev); bad += run<4, 2>(3, rev); bad += run<5, 2>(4, rev);
        bad += run<6, 2>(5, rev); bad += run<7, 1>(6, rev); bad += run<2, 1>(7, rev); bad += run<3, 2>(8, rev);
        bad += run<4, 1>(9, rev); bad += run<5, 1>(10, rev);
    }
    printf(bad == 0 ? "ALL OK\n" : "FAILURES\n");
    return bad == 0 ? 0 : 1;
}
