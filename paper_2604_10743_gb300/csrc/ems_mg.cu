// ems_mg.cu -- smoothed-aggregation multigrid preconditioner for the IR-drop
// PCG (Sec. III-C, Eq. ir_drop_mna is solved by CG; the preconditioner is
// this library's choice).
//
// Setup (host, once per grid, from the initial resistances): greedy
// aggregation of the conductance graph (strong couplings |a_ij| >=
// 0.08 sqrt(a_ii a_jj)), tentative piecewise-constant prolongation smoothed
// by one damped-Jacobi step, P = (I - omega D^-1 A) P_tent with
// omega = 4 / (3 rho), rho the Gershgorin bound of D^-1 A, Galerkin coarse
// operators P^T A P, down to <= 512 unknowns, where the dense inverse is
// formed by Cholesky.  The hierarchy depends only on the grid and R0: voids
// change a few resistances by small factors and Monte Carlo factors do not
// touch R, so one hierarchy serves every sample for the whole run, while the
// finest level always uses the current matrix.
//
// Application (device): one symmetric V(1,1) cycle with damped-Jacobi
// smoothing (2/3), which keeps the preconditioner symmetric positive
// definite.  Two kernels: one CTA per sample for systems of <= 4,096
// unknowns; a cooperative grid for larger ones, where the levels above 1,024
// unknowns (MGDevice::small) run grid-wide between bounded grid barriers and
// block 0 runs the small levels alone.  All sums are fixed-order (bitwise reproducible).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include <cooperative_groups.h>

#include "ems_internal.cuh"

namespace cg = cooperative_groups;

namespace ems {

namespace {

constexpr double kStrength = 0.08;
constexpr int kCoarsest = 512;
constexpr double kSmooth = 2.0 / 3.0;   // damped-Jacobi weight of the V-cycle

struct SpM {
    int nr = 0, nc = 0;
    std::vector<int32_t> ptr, col;
    std::vector<double> val;
};

SpM transpose(const SpM &A) {
    SpM T;
    T.nr = A.nc; T.nc = A.nr;
    T.ptr.assign(T.nr + 1, 0);
    for (int32_t c : A.col) ++T.ptr[c + 1];
    for (int i = 0; i < T.nr; ++i) T.ptr[i + 1] += T.ptr[i];
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    std::vector<int32_t> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int r = 0; r < A.nr; ++r)
        for (int k = A.ptr[r]; k < A.ptr[r + 1]; ++k) {
            const int q = fill[A.col[k]]++;
            T.col[q] = r;
            T.val[q] = A.val[k];
        }
    return T;   // rows come out with ascending columns
}

// rows [0, nr) built in parallel blocks: row(i, acc, mark, cols, col, val)
// appends row i to (col, val) using the block's own scratch; the blocks are
// concatenated in order, so every row's sums run in the same order as a
// serial pass (the result is the same bit for bit)
template <class Row>
SpM build_rows(int nr, int nc, Row row) {
    const int nblk = std::max(1, std::min(256, nr / 4096));
    std::vector<std::vector<int32_t>> bptr(nblk), bcol(nblk);
    std::vector<std::vector<double>> bval(nblk);
    parallel_for(nblk, [&](int q) {
        const int r0 = (int)((int64_t)nr * q / nblk), r1 = (int)((int64_t)nr * (q + 1) / nblk);
        std::vector<double> acc(nc, 0.0);
        std::vector<int32_t> mark(nc, -1), cols;
        auto &pp = bptr[q];
        pp.reserve(r1 - r0);
        for (int i = r0; i < r1; ++i) {
            row(i, acc, mark, cols, bcol[q], bval[q]);
            pp.push_back((int32_t)bcol[q].size());
        }
    });
    SpM C;
    C.nr = nr; C.nc = nc;
    C.ptr.assign(1, 0);
    size_t tot = 0;
    for (int q = 0; q < nblk; ++q) tot += bcol[q].size();
    C.ptr.reserve(nr + 1); C.col.reserve(tot); C.val.reserve(tot);
    for (int q = 0; q < nblk; ++q) {
        const int32_t o = (int32_t)C.col.size();
        for (int32_t v : bptr[q]) C.ptr.push_back(o + v);
        C.col.insert(C.col.end(), bcol[q].begin(), bcol[q].end());
        C.val.insert(C.val.end(), bval[q].begin(), bval[q].end());
    }
    return C;
}

SpM spmm(const SpM &A, const SpM &B) {
    return build_rows(A.nr, B.nc, [&](int i, std::vector<double> &acc, std::vector<int32_t> &mark,
                                       std::vector<int32_t> &cols, std::vector<int32_t> &ocol,
                                       std::vector<double> &oval) {
        cols.clear();
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            const double a = A.val[k];
            const int r = A.col[k];
            for (int m = B.ptr[r]; m < B.ptr[r + 1]; ++m) {
                const int c = B.col[m];
                if (mark[c] != i) { mark[c] = i; acc[c] = 0.0; cols.push_back(c); }
                acc[c] += a * B.val[m];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int c : cols) { ocol.push_back(c); oval.push_back(acc[c]); }
    });
}

std::vector<double> diagonal(const SpM &A) {
    std::vector<double> d(A.nr, 0.0);
    for (int i = 0; i < A.nr; ++i)
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (A.col[k] == i) d[i] += A.val[k];
    return d;
}

// greedy aggregation; returns the aggregate of every row and their number
std::vector<int32_t> aggregate(const SpM &A, const std::vector<double> &d, int &nagg) {
    const int n = A.nr;
    auto strong = [&](int i, int k) {
        const int j = A.col[k];
        return j != i && std::fabs(A.val[k]) >= kStrength * std::sqrt(d[i] * d[j]);
    };
    std::vector<int32_t> agg(n, -1);
    nagg = 0;
    // pass 1: a row whose strong neighbours are all free seeds an aggregate
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        bool free = true;
        for (int k = A.ptr[i]; k < A.ptr[i + 1] && free; ++k)
            if (strong(i, k) && agg[A.col[k]] >= 0) free = false;
        if (!free) continue;
        agg[i] = nagg;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (strong(i, k)) agg[A.col[k]] = nagg;
        ++nagg;
    }
    // pass 2: join the aggregate of the strongest pass-1 neighbour
    const std::vector<int32_t> first = agg;
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        double best = 0.0;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            if (strong(i, k) && first[A.col[k]] >= 0 && std::fabs(A.val[k]) > best) {
                best = std::fabs(A.val[k]);
                agg[i] = first[A.col[k]];
            }
    }
    // pass 3: rows left alone form their own aggregates
    for (int i = 0; i < n; ++i)
        if (agg[i] < 0) agg[i] = nagg++;
    return agg;
}

// P = (I - omega D^-1 A) P_tent
SpM smoothed_prolongation(const SpM &A, const std::vector<double> &d, const std::vector<int32_t> &agg, int nagg) {
    double rho = 0.0;
    for (int i = 0; i < A.nr; ++i) {
        double s = 0.0;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += std::fabs(A.val[k]);
        rho = std::max(rho, s / d[i]);
    }
    const double omega = 4.0 / (3.0 * rho);
    return build_rows(A.nr, nagg, [&](int i, std::vector<double> &acc, std::vector<int32_t> &mark,
                                      std::vector<int32_t> &cols, std::vector<int32_t> &ocol,
                                      std::vector<double> &oval) {
        cols.clear();
        auto add = [&](int c, double v) {
            if (mark[c] != i) { mark[c] = i; acc[c] = 0.0; cols.push_back(c); }
            acc[c] += v;
        };
        add(agg[i], 1.0);
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) add(agg[A.col[k]], -omega * A.val[k] / d[i]);
        std::sort(cols.begin(), cols.end());
        for (int c : cols)
            if (acc[c] != 0.0) { ocol.push_back(c); oval.push_back(acc[c]); }
    });
}

// inverse of an SPD dense matrix by Cholesky; false if not positive definite.
// The rows below each pivot and the columns of the inverse run on the host's
// cores; every entry's sums keep their order (the same result as one core).
bool spd_inverse(int n, std::vector<double> &a /* n x n, in: A, out: A^-1 */) {
    std::vector<double> L((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = a[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        const int rows = n - j - 1;
        const int nb = std::max(1, std::min(64, rows / 64));
        parallel_for(nb, [&](int q) {
            const int i0 = j + 1 + (int)((int64_t)rows * q / nb), i1 = j + 1 + (int)((int64_t)rows * (q + 1) / nb);
            for (int i = i0; i < i1; ++i) {
                double t = a[(size_t)i * n + j];
                for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
                L[(size_t)i * n + j] = t / ljj;
            }
        });
    }
    std::vector<double> LT((size_t)n * n);              // LT[i][k] = L[k][i]
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) LT[(size_t)i * n + k] = L[(size_t)k * n + i];
    parallel_for(n, [&](int c) {
        std::vector<double> y(n, 0.0), x(n);
        for (int i = c; i < n; ++i) {                    // L y = e_c (y_i = 0 for i < c)
            double t = i == c ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) t -= L[(size_t)i * n + k] * y[k];
            y[i] = t / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {               // L^T x = y
            double t = y[i];
            for (int k = i + 1; k < n; ++k) t -= LT[(size_t)i * n + k] * x[k];
            x[i] = t / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) a[(size_t)i * n + c] = x[i];
    });
    return true;
}

}  // namespace

// Builds the hierarchy of the free-node conductance matrix with values from
// R0.  Leaves h.L = 0 (Jacobi only) when the system is small or coarsening
// stalls.
void mg_build(int nf, const std::vector<int32_t> &ptr, const std::vector<int32_t> &col,
              const std::vector<int32_t> &ent_ptr, const std::vector<int32_t> &ent_seg,
              const std::vector<int8_t> &ent_diag, const double *R0, int min_rows, MGHost &h) {
    h = MGHost();
    if (nf < min_rows || nf < 2 * kCoarsest) return;
    SpM A;
    A.nr = A.nc = nf;
    A.ptr = ptr;
    A.col = col;
    A.val.resize(col.size());
    for (size_t k = 0; k < col.size(); ++k) {
        double v = 0.0;
        for (int e = ent_ptr[k]; e < ent_ptr[k + 1]; ++e) v += 1.0 / R0[ent_seg[e]];
        A.val[k] = ent_diag[k] ? v : -v;
    }
    std::vector<SpM> As{A}, Ps, Rs;
    std::vector<std::vector<double>> Ds{diagonal(A)};
    while (As.back().nr > kCoarsest && (int)As.size() < EMS_MG_MAXLV) {
        const SpM &Al = As.back();
        int nagg = 0;
        const std::vector<int32_t> agg = aggregate(Al, Ds.back(), nagg);
        if (nagg > 0.8 * Al.nr) break;           // coarsening stalled
        SpM P = smoothed_prolongation(Al, Ds.back(), agg, nagg);
        SpM R = transpose(P);
        SpM Ac = spmm(R, spmm(Al, P));
        Ps.push_back(std::move(P));
        Rs.push_back(std::move(R));
        Ds.push_back(diagonal(Ac));
        As.push_back(std::move(Ac));
    }
    const int nc = As.back().nr;
    if (As.size() < 2 || nc > 4 * kCoarsest) return;
    std::vector<double> dense((size_t)nc * nc, 0.0);
    for (int i = 0; i < nc; ++i)
        for (int k = As.back().ptr[i]; k < As.back().ptr[i + 1]; ++k)
            dense[(size_t)i * nc + As.back().col[k]] += As.back().val[k];
    if (!spd_inverse(nc, dense)) return;
    // flatten: ints [A ptr, A col (levels >= 1), P ptr, P col, R ptr, R col
    // (levels < L-1)], doubles [A val, dinv (levels >= 1), P val, R val, C^-1]
    const int L = (int)As.size();
    h.L = L;
    auto put_i = [&](const std::vector<int32_t> &v) {
        const int64_t o = (int64_t)h.ints.size();
        h.ints.insert(h.ints.end(), v.begin(), v.end());
        while (h.ints.size() % 64) h.ints.push_back(0);
        return o;
    };
    auto put_d = [&](const std::vector<double> &v) {
        const int64_t o = (int64_t)h.dbls.size();
        h.dbls.insert(h.dbls.end(), v.begin(), v.end());
        while (h.dbls.size() % 32) h.dbls.push_back(0.0);
        return o;
    };
    int64_t sc = 0;
    for (int l = 0; l < L; ++l) {
        MGLevelDesc &d = h.lv[l];
        d.n = As[l].nr;
        if (l > 0) {
            d.a_ptr = put_i(As[l].ptr);
            d.a_col = put_i(As[l].col);
            d.a_val = put_d(As[l].val);
            std::vector<double> di(Ds[l].size());
            for (size_t i = 0; i < di.size(); ++i) di[i] = 1.0 / Ds[l][i];
            d.dinv = put_d(di);
        }
        if (l + 1 < L) {
            d.p_ptr = put_i(Ps[l].ptr);
            d.p_col = put_i(Ps[l].col);
            d.p_val = put_d(Ps[l].val);
            d.r_ptr = put_i(Rs[l].ptr);
            d.r_col = put_i(Rs[l].col);
            d.r_val = put_d(Rs[l].val);
        }
        // per-sample scratch: e and t on every level, r below the finest
        auto align = [](int64_t x) { return (x + 31) / 32 * 32; };
        d.e = sc; sc = align(sc + d.n);
        d.t = sc; sc = align(sc + d.n);
        if (l > 0) { d.r = sc; sc = align(sc + d.n); }
        h.nnz += (int64_t)As[l].col.size();
    }
    h.cinv = put_d(dense);
    h.per_sample = sc;
}

namespace {

constexpr int kStatusNoConv = 0;
constexpr int kStatusTimeout = 1;

struct MGArgs {
    int nf, S;
    int64_t nnz;
    const int32_t *ptr, *col;                   // finest level structure
    const double *val, *b, *dinv;               // [S][nnz], [S][nf], [S][nf]
    double *x, *r, *p, *q, *z;                  // [S][nf]
    const float *val32, *dinv32;                // the finest level in FP32 (FP32 V-cycle)
    float *r32;                                 // [S][nf] the residual rounded to FP32 (V-cycle input)
    double rtol;
    int max_iter;
    int32_t *iters, *status;
    double *red;
    unsigned int *bar;
    MGDevice g;
};

template <int K>
__device__ void bsum(double (&v)[K], double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) sh[q * 32 + w] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += sh[q * 32 + k];
        v[q] = t;
    }
}

__device__ bool gsync(unsigned int *bar, int32_t *status) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = bar + 1;
        const long long limit = *((volatile long long *)(bar + 2));   // polls before giving up
        const unsigned int gen = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long spins = 0;
            while (*vgen == gen) {
                if (++spins > limit || *((volatile int32_t *)&status[kStatusTimeout])) {
                    atomicOr(&status[kStatusTimeout], 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <int K>
__device__ bool gsum(double (&v)[K], double *sh, double *red, unsigned int *bar, int32_t *status) {
    __shared__ double bc[K];
    bsum<K>(v, sh);
    const int G = gridDim.x;
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) red[q * G + blockIdx.x] = v[q];
    __threadfence();
    if (!gsync(bar, status)) return false;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = 0.0;
            for (int k = threadIdx.x; k < G; k += 32) t += __ldcg(red + q * G + k);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (threadIdx.x == 0) bc[q] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = bc[q];
    return true;
}

// The V-cycle's arithmetic type P: double in FP64 contexts; float in FP32
// ones, from an FP32 copy of the hierarchy and of the finest matrix, with the
// CG iteration itself (matrix products, residual, dot products, the
// convergence test) in FP64 -- the mixed-precision form: FP64 only where the
// residual is formed.  A preconditioner rounded to FP32 is not exactly
// linear, so the FP32 variants take the flexible (Polak-Ribiere) beta,
// (r_new.z_new - r_new.z_old) / (r_old.z_old), which keeps CG convergent
// with a slightly varying preconditioner.
template <typename P> __device__ __forceinline__ const P *hier(const MGArgs &a);
template <> __device__ __forceinline__ const double *hier<double>(const MGArgs &a) { return a.g.D; }
template <> __device__ __forceinline__ const float *hier<float>(const MGArgs &a) { return a.g.F; }

template <typename P>
__device__ __forceinline__ P csr_dot(const int32_t *ptr, const int32_t *col, const P *val, const P *v, int i) {
    P acc = P(0);
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) acc += val[k] * v[col[k]];
    return acc;
}

// one level's operators: the finest uses the current matrix of the sample
template <typename P>
struct Lv {
    int n;
    const int32_t *ap, *ac;
    const P *av, *dv;
};

template <typename P>
__device__ __forceinline__ Lv<P> level(const MGArgs &a, const P *val0, const P *dinv0, int l) {
    const MGLevelDesc &d = a.g.lv[l];
    if (l == 0) return Lv<P>{a.nf, a.ptr, a.col, val0, dinv0};
    return Lv<P>{d.n, a.g.I + d.a_ptr, a.g.I + d.a_col, hier<P>(a) + d.a_val, hier<P>(a) + d.dinv};
}

// Phase sequence of the V-cycle from level l0 (input r_l0) over the rows
// [start, n) in steps of `stride`, with `sync` between phases.  Level l's
// result lands in t_l; the coarsest level's in e.  fused: the caller has
// already set e_l0 = w D^-1 r_l0, and each restriction also sets the next
// level's e (the pre-smoothing needs no phase of its own).
template <typename P, class Sync>
__device__ bool vcycle(const MGArgs &a, const P *val0, const P *dinv0, P *sc, int l0, int l1, const P *r_l0,
                       int start, int stride, Sync sync, bool fused = false) {
    const int L = a.g.L;
    const P *r = r_l0;
    const P w = P(kSmooth);
    for (int l = l0; l < l1 && l < L - 1; ++l) {
        const Lv<P> A = level<P>(a, val0, dinv0, l);
        const MGLevelDesc &d = a.g.lv[l];
        P *e = sc + d.e, *t = sc + d.t;
        if (!fused) {
            for (int i = start; i < A.n; i += stride) e[i] = w * A.dv[i] * r[i];
            if (!sync()) return false;
        }
        for (int i = start; i < A.n; i += stride) t[i] = r[i] - csr_dot<P>(A.ap, A.ac, A.av, e, i);
        if (!sync()) return false;
        const MGLevelDesc &dn = a.g.lv[l + 1];
        P *rn = sc + dn.r;
        const int32_t *rp = a.g.I + d.r_ptr, *rc = a.g.I + d.r_col;
        const P *rv = hier<P>(a) + d.r_val;
        if (fused && l + 1 < L - 1) {
            const P *dvn = hier<P>(a) + dn.dinv;
            P *en = sc + dn.e;
            for (int i = start; i < dn.n; i += stride) {
                const P v = csr_dot<P>(rp, rc, rv, t, i);
                rn[i] = v;
                en[i] = w * dvn[i] * v;
            }
        } else {
            for (int i = start; i < dn.n; i += stride) rn[i] = csr_dot<P>(rp, rc, rv, t, i);
        }
        if (!sync()) return false;
        r = rn;
    }
    return true;
}

// Up sweep from level l_hi down to l_lo; level l0's result goes to out
// (type O: the FP64 z at the finest level, scratch above it).  acc
// (optional): the last phase also accumulates r.z and r.r of the rows it
// writes into acc[0], acc[1] (r from racc, the FP64 residual) and leaves the
// closing barrier to the caller.
template <typename P, typename O, class Sync>
__device__ bool vcycle_up(const MGArgs &a, const P *val0, const P *dinv0, P *sc, int l_hi, int l_lo,
                          const P *r_l0, O *out, int l0, int start, int stride, Sync sync, double *acc = nullptr,
                          const double *racc = nullptr) {
    const int L = a.g.L;
    const P w = P(kSmooth);
    for (int l = l_hi; l >= l_lo; --l) {
        const Lv<P> A = level<P>(a, val0, dinv0, l);
        const MGLevelDesc &d = a.g.lv[l], &dn = a.g.lv[l + 1];
        const P *en = (l + 1 == L - 1) ? sc + dn.e : sc + dn.t;
        P *e = sc + d.e;
        const int32_t *pp = a.g.I + d.p_ptr, *pc = a.g.I + d.p_col;
        const P *pv = hier<P>(a) + d.p_val;
        for (int i = start; i < A.n; i += stride) e[i] += csr_dot<P>(pp, pc, pv, en, i);
        if (!sync()) return false;
        const P *rl = l == l0 ? r_l0 : sc + d.r;
        if (l == l0) {
            if (acc && l == l_lo) {
                for (int i = start; i < A.n; i += stride) {
                    const O oi = (O)(e[i] + w * A.dv[i] * (rl[i] - csr_dot<P>(A.ap, A.ac, A.av, e, i)));
                    out[i] = oi;
                    acc[0] += racc[i] * (double)oi;
                    acc[1] += racc[i] * racc[i];
                }
                continue;
            }
            for (int i = start; i < A.n; i += stride)
                out[i] = (O)(e[i] + w * A.dv[i] * (rl[i] - csr_dot<P>(A.ap, A.ac, A.av, e, i)));
        } else {
            P *o = sc + d.t;
            for (int i = start; i < A.n; i += stride)
                o[i] = e[i] + w * A.dv[i] * (rl[i] - csr_dot<P>(A.ap, A.ac, A.av, e, i));
        }
        if (!sync()) return false;
    }
    return true;
}

// coarsest level: e_c = C^-1 r_c
template <typename P, class Sync>
__device__ bool coarse(const MGArgs &a, P *sc, int start, int stride, Sync sync) {
    const int L = a.g.L;
    const MGLevelDesc &d = a.g.lv[L - 1];
    const int n = d.n;
    const P *ci = hier<P>(a) + a.g.cinv, *r = sc + d.r;
    P *e = sc + d.e;
    for (int i = start; i < n; i += stride) {
        P acc = P(0);
        for (int j = 0; j < n; ++j) acc += ci[(size_t)i * n + j] * r[j];
        e[i] = acc;
    }
    return sync();
}

// whole V-cycle in one CTA: z = M^-1 r
template <typename P>
__device__ void vcycle_block(const MGArgs &a, const P *val0, const P *dinv0, P *sc, const P *r, double *z) {
    auto bs = []() { __syncthreads(); return true; };
    const int L = a.g.L;
    vcycle<P>(a, val0, dinv0, sc, 0, L - 1, r, threadIdx.x, blockDim.x, bs);
    coarse<P>(a, sc, threadIdx.x, blockDim.x, bs);
    vcycle_up<P>(a, val0, dinv0, sc, L - 2, 0, r, z, 0, threadIdx.x, blockDim.x, bs);
}

// the sample's finest-level operators and V-cycle input in the type P
template <typename P> struct Fine;
template <> struct Fine<double> {
    const double *val, *dinv;
    double *rin;
    __device__ Fine(const MGArgs &a, int s)
        : val(a.val + (size_t)s * a.nnz), dinv(a.dinv + (size_t)s * a.nf), rin(a.r + (size_t)s * a.nf) {}
    __device__ void set(int, double) const {}            // the input is r itself
};
template <> struct Fine<float> {
    const float *val, *dinv;
    float *rin;
    __device__ Fine(const MGArgs &a, int s)
        : val(a.val32 + (size_t)s * a.nnz), dinv(a.dinv32 + (size_t)s * a.nf), rin(a.r32 + (size_t)s * a.nf) {}
    __device__ void set(int i, double ri) const { rin[i] = (float)ri; }
};
template <typename P> constexpr bool kFlexible = sizeof(P) == 4;

// Mode A with the multigrid preconditioner: one CTA per sample
template <typename P>
__global__ void __launch_bounds__(1024) k_pcg_block_mg(MGArgs a) {
    __shared__ double sh[96];
    const int s = blockIdx.x, nf = a.nf;
    const double *val = a.val + (size_t)s * a.nnz, *b = a.b + (size_t)s * nf;
    double *x = a.x + (size_t)s * nf, *r = a.r + (size_t)s * nf, *p = a.p + (size_t)s * nf;
    double *q = a.q + (size_t)s * nf, *z = a.z + (size_t)s * nf;
    P *sc = reinterpret_cast<P *>(a.g.scratch + (size_t)s * a.g.per_sample);
    const Fine<P> fn(a, s);
    double v2[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const double ri = b[i] - csr_dot<double>(a.ptr, a.col, val, x, i);
        r[i] = ri;
        fn.set(i, ri);
        v2[0] += ri * ri;
        v2[1] += b[i] * b[i];
    }
    bsum<2>(v2, sh);
    double rr = v2[0];
    const double tol2 = a.rtol * a.rtol * v2[1];
    int it = 0;
    double rz = 0.0;
    if (rr > tol2) {
        vcycle_block<P>(a, fn.val, fn.dinv, sc, fn.rin, z);
        double v1[1] = {0.0};
        for (int i = threadIdx.x; i < nf; i += blockDim.x) { p[i] = z[i]; v1[0] += r[i] * z[i]; }
        bsum<1>(v1, sh);
        rz = v1[0];
    }
    while (rr > tol2 && it < a.max_iter) {
        __syncthreads();
        double v1[1] = {0.0};
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            const double qi = csr_dot<double>(a.ptr, a.col, val, p, i);
            q[i] = qi;
            v1[0] += p[i] * qi;
        }
        bsum<1>(v1, sh);
        const double alpha = rz / v1[0];
        double rzo = 0.0;                              // r_new . z_old (flexible beta)
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            fn.set(i, r[i]);
            if (kFlexible<P>) rzo += r[i] * z[i];
        }
        __syncthreads();
        vcycle_block<P>(a, fn.val, fn.dinv, sc, fn.rin, z);
        double w2[3] = {0.0, 0.0, rzo};
        for (int i = threadIdx.x; i < nf; i += blockDim.x) { w2[0] += r[i] * z[i]; w2[1] += r[i] * r[i]; }
        if (kFlexible<P>) bsum<3>(w2, sh);
        else bsum<2>(reinterpret_cast<double (&)[2]>(w2), sh);
        const double beta = (kFlexible<P> ? w2[0] - w2[2] : w2[0]) / rz;
        rz = w2[0];
        rr = w2[1];
        for (int i = threadIdx.x; i < nf; i += blockDim.x) p[i] = z[i] + beta * p[i];
        ++it;
    }
    if (threadIdx.x == 0) {
        a.iters[s] = it;
        if (rr > tol2) atomicOr(&a.status[kStatusNoConv], 1);
    }
}

// grid-wide V-cycle: large levels across the grid, small ones in block 0.
// The caller has set e_0 = w D^-1 r (fused pre-smoothing); with acc the last
// phase accumulates (r.z, r.r) and the caller's reduction closes it.
template <typename P>
__device__ bool vcycle_grid(const MGArgs &a, const P *val0, const P *dinv0, P *sc, const P *r, double *z,
                            double *acc, const double *racc) {
    const int L = a.g.L;
    int lb = 0;                       // first level small enough for one CTA
    while (lb < L - 1 && a.g.lv[lb].n > a.g.small) ++lb;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    auto gsy = [&]() { return gsync(a.bar, a.status); };
    auto bs = []() { __syncthreads(); return true; };
    if (!vcycle<P>(a, val0, dinv0, sc, 0, lb, r, gid, gs, gsy, true)) return false;
    if (blockIdx.x == 0) {
        // levels lb..L-1 in this CTA; level lb's input sits in its r slot
        // (lb > 0 always: the finest level is above the small threshold)
        const P *rl = sc + a.g.lv[lb].r;
        P *ol = sc + a.g.lv[lb].t;
        vcycle<P>(a, val0, dinv0, sc, lb, L - 1, rl, threadIdx.x, blockDim.x, bs, true);
        coarse<P>(a, sc, threadIdx.x, blockDim.x, bs);
        if (lb <= L - 2) vcycle_up<P>(a, val0, dinv0, sc, L - 2, lb, rl, ol, lb, threadIdx.x, blockDim.x, bs);
        __threadfence();
    }
    if (!gsy()) return false;
    return vcycle_up<P>(a, val0, dinv0, sc, lb - 1, 0, r, z, 0, gid, gs, gsy, acc, racc);
}

// Mode B with the multigrid preconditioner: cooperative grid, samples in turn
template <typename P>
__global__ void __launch_bounds__(512, 2) k_pcg_grid_mg(MGArgs a) {
    __shared__ double sh[96];
    const int nf = a.nf, G = gridDim.x;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gs = G * blockDim.x;
    double *redA = a.red, *redB = a.red + 3 * G;
    const P w = P(kSmooth);
    for (int s = 0; s < a.S; ++s) {
        const double *val = a.val + (size_t)s * a.nnz, *b = a.b + (size_t)s * nf;
        double *x = a.x + (size_t)s * nf, *r = a.r + (size_t)s * nf, *p = a.p + (size_t)s * nf;
        double *q = a.q + (size_t)s * nf, *z = a.z + (size_t)s * nf;
        P *sc = reinterpret_cast<P *>(a.g.scratch + (size_t)s * a.g.per_sample);
        const Fine<P> fn(a, s);
        P *e0 = sc + a.g.lv[0].e;                  // pre-smoothing of the V-cycle, fused below
        double v2[2] = {0.0, 0.0};
        for (int i = gid; i < nf; i += gs) {
            const double ri = b[i] - csr_dot<double>(a.ptr, a.col, val, x, i);
            r[i] = ri;
            fn.set(i, ri);
            e0[i] = w * fn.dinv[i] * (P)ri;
            v2[0] += ri * ri;
            v2[1] += b[i] * b[i];
        }
        if (!gsum<2>(v2, sh, redA, a.bar, a.status)) return;
        double rr = v2[0];
        const double tol2 = a.rtol * a.rtol * v2[1];
        int it = 0;
        double rz = 0.0;
        if (rr > tol2) {
            if (!vcycle_grid<P>(a, fn.val, fn.dinv, sc, fn.rin, z, nullptr, r)) return;
            double v1[1] = {0.0};
            for (int i = gid; i < nf; i += gs) { p[i] = z[i]; v1[0] += r[i] * z[i]; }
            if (!gsum<1>(v1, sh, redB, a.bar, a.status)) return;
            rz = v1[0];
        }
        while (rr > tol2 && it < a.max_iter) {
            double v1[1] = {0.0};
            for (int i = gid; i < nf; i += gs) {
                const double qi = csr_dot<double>(a.ptr, a.col, val, p, i);
                q[i] = qi;
                v1[0] += p[i] * qi;
            }
            if (!gsum<1>(v1, sh, redA, a.bar, a.status)) return;
            const double alpha = rz / v1[0];
            double rzo = 0.0;                          // r_new . z_old (flexible beta)
            for (int i = gid; i < nf; i += gs) {
                x[i] += alpha * p[i];
                const double ri = r[i] - alpha * q[i];
                r[i] = ri;
                fn.set(i, ri);
                e0[i] = w * fn.dinv[i] * (P)ri;
                if (kFlexible<P>) rzo += ri * z[i];
            }
            if (!gsync(a.bar, a.status)) return;          // r, e0 complete
            double w2[3] = {0.0, 0.0, rzo};
            if (!vcycle_grid<P>(a, fn.val, fn.dinv, sc, fn.rin, z, w2, r)) return;
            if (kFlexible<P>) {
                if (!gsum<3>(w2, sh, redB, a.bar, a.status)) return;
            } else {
                if (!gsum<2>(reinterpret_cast<double (&)[2]>(w2), sh, redB, a.bar, a.status)) return;
            }
            const double beta = (kFlexible<P> ? w2[0] - w2[2] : w2[0]) / rz;
            rz = w2[0];
            rr = w2[1];
            for (int i = gid; i < nf; i += gs) p[i] = z[i] + beta * p[i];
            if (!gsync(a.bar, a.status)) return;          // p complete
            ++it;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.iters[s] = it;
            if (rr > tol2) atomicOr(&a.status[kStatusNoConv], 1);
        }
        if (!gsync(a.bar, a.status)) return;
    }
}

// Mode C: one thread-block cluster per sample, for several samples at once
// (one sample is faster on the whole grid: 16 SMs cannot hide the gather
// latency of the finest level).  Cluster barriers are hardware barriers (no
// spin), sums go through distributed shared memory in rank order, and every
// level of the V-cycle runs across the cluster.
template <int K>
__device__ void csum(double (&v)[K], double *sh, double *slot, cg::cluster_group &cl) {
    bsum<K>(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) slot[q] = v[q];
    cl.sync();
    const int CL = (int)cl.num_blocks();
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = 0.0;
    for (int r = 0; r < CL; ++r) {
        const double *o = cl.map_shared_rank(slot, r);
#pragma unroll
        for (int q = 0; q < K; ++q) v[q] += o[q];
    }
}

template <typename P>
__global__ void __launch_bounds__(1024) k_pcg_cluster_mg(MGArgs a) {
    __shared__ double sh[96];
    __shared__ double slots[2][4];                 // alternate so a slot is not rewritten while read
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int s = blockIdx.x / CL, nf = a.nf;
    const int gid = rank * blockDim.x + threadIdx.x, gs = CL * blockDim.x;
    const double *val = a.val + (size_t)s * a.nnz, *b = a.b + (size_t)s * nf;
    double *x = a.x + (size_t)s * nf, *r = a.r + (size_t)s * nf, *p = a.p + (size_t)s * nf;
    double *q = a.q + (size_t)s * nf, *z = a.z + (size_t)s * nf;
    P *sc = reinterpret_cast<P *>(a.g.scratch + (size_t)s * a.g.per_sample);
    const Fine<P> fn(a, s);
    auto csy = [&]() { cl.sync(); return true; };
    const int L = a.g.L;
    auto vcyc = [&]() {
        vcycle<P>(a, fn.val, fn.dinv, sc, 0, L - 1, fn.rin, gid, gs, csy);
        coarse<P>(a, sc, gid, gs, csy);
        vcycle_up<P>(a, fn.val, fn.dinv, sc, L - 2, 0, fn.rin, z, 0, gid, gs, csy);
    };
    int par = 0;
    double v2[2] = {0.0, 0.0};
    for (int i = gid; i < nf; i += gs) {
        const double ri = b[i] - csr_dot<double>(a.ptr, a.col, val, x, i);
        r[i] = ri;
        fn.set(i, ri);
        v2[0] += ri * ri;
        v2[1] += b[i] * b[i];
    }
    csum<2>(v2, sh, slots[par], cl); par ^= 1;
    double rr = v2[0];
    const double tol2 = a.rtol * a.rtol * v2[1];
    int it = 0;
    double rz = 0.0;
    if (rr > tol2) {
        cl.sync();                                     // r complete
        vcyc();
        double v1[1] = {0.0};
        for (int i = gid; i < nf; i += gs) { p[i] = z[i]; v1[0] += r[i] * z[i]; }
        csum<1>(v1, sh, slots[par], cl); par ^= 1;     // also: p complete
        rz = v1[0];
    }
    while (rr > tol2 && it < a.max_iter) {
        double v1[1] = {0.0};
        for (int i = gid; i < nf; i += gs) {
            const double qi = csr_dot<double>(a.ptr, a.col, val, p, i);
            q[i] = qi;
            v1[0] += p[i] * qi;
        }
        csum<1>(v1, sh, slots[par], cl); par ^= 1;
        const double alpha = rz / v1[0];
        double rzo = 0.0;                              // r_new . z_old (flexible beta)
        for (int i = gid; i < nf; i += gs) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            fn.set(i, r[i]);
            if (kFlexible<P>) rzo += r[i] * z[i];
        }
        cl.sync();                                     // r complete
        vcyc();
        double w2[3] = {0.0, 0.0, rzo};
        for (int i = gid; i < nf; i += gs) { w2[0] += r[i] * z[i]; w2[1] += r[i] * r[i]; }
        if (kFlexible<P>) csum<3>(w2, sh, slots[par], cl);
        else csum<2>(reinterpret_cast<double (&)[2]>(w2), sh, slots[par], cl);
        par ^= 1;
        const double beta = (kFlexible<P> ? w2[0] - w2[2] : w2[0]) / rz;
        rz = w2[0];
        rr = w2[1];
        for (int i = gid; i < nf; i += gs) p[i] = z[i] + beta * p[i];
        cl.sync();                                     // p complete
        ++it;
    }
    if (rank == 0 && threadIdx.x == 0) {
        a.iters[s] = it;
        if (rr > tol2) atomicOr(&a.status[kStatusNoConv], 1);
    }
    cl.sync();                                         // no CTA leaves while its slots may be read
}

}  // namespace

// PCG with the multigrid preconditioner (the hierarchy must exist); the
// V-cycle in the context's stress precision
template <typename P>
ems_status mg_solve_t(ems_ctx *c) {
    Dev &d = c->d;
    cudaStream_t st = c->stream;
    MGArgs a;
    a.nf = c->nf; a.S = c->S; a.nnz = c->nnz;
    a.ptr = d.csr_ptr; a.col = d.csr_col; a.val = d.csr_val; a.b = d.ir_b; a.dinv = d.ir_dinv;
    a.x = d.ir_x; a.r = d.ir_r; a.p = d.ir_p; a.q = d.ir_Ap; a.z = d.ir_z;
    a.val32 = d.val32; a.dinv32 = d.dinv32; a.r32 = d.r32;
    a.rtol = c->prm.ir_rtol; a.max_iter = c->prm.ir_max_iter;
    a.iters = d.ir_iters; a.status = d.status; a.red = d.red; a.bar = d.gbar;
    a.g = c->mg;
    if (c->nf <= 4096) {
        const int threads = c->nf >= 1024 ? 1024 : ((c->nf + 31) / 32) * 32;
        k_pcg_block_mg<P><<<c->S, threads, 0, st>>>(a);
        ++c->launches;
        EMS_CUDA(c, cudaGetLastError());
        return EMS_OK;
    }
    // one cluster per sample when the device can hold one of 16 (or 8) CTAs
    if (c->mg_cluster == 0) {
        c->mg_cluster = -1;
        if (cudaFuncSetAttribute(k_pcg_cluster_mg<P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
            cudaGetLastError();
        for (int cs : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(cs); cfg.blockDim = dim3(1024); cfg.attrs = at; cfg.numAttrs = 1;
            int nclus = 0;
            if (cudaOccupancyMaxActiveClusters(&nclus, k_pcg_cluster_mg<P>, &cfg) == cudaSuccess && nclus > 0) {
                c->mg_cluster = cs;
                break;
            }
            cudaGetLastError();
        }
    }
    if (c->mg_cluster > 0 && c->S > 1) {              // samples as parallel clusters
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = c->mg_cluster; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(c->mg_cluster * c->S); cfg.blockDim = dim3(1024); cfg.stream = st;
        cfg.attrs = at; cfg.numAttrs = 1;
        EMS_CUDA(c, cudaLaunchKernelEx(&cfg, k_pcg_cluster_mg<P>, a));
        ++c->launches;
        return EMS_OK;
    }
    if (c->mg_blocks == 0) {
        int dev = 0, nsm = 0, per = 0;
        EMS_CUDA(c, cudaGetDevice(&dev));
        EMS_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        EMS_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_grid_mg<P>, 512, 0));
        if (per < 1) return fail(c, EMS_E_CUDA, "cooperative multigrid PCG cannot be resident");
        const int need = (c->nf + 511) / 512;
        int G = nsm * (per < 2 ? per : 2);
        if (G > need) G = need;
        if (G > 680) G = 680;                         // red[] holds 2 x 3 partials per block
        c->mg_blocks = G;
    }
    EMS_CUDA(c, cudaMemsetAsync(d.gbar, 0, 2 * sizeof(unsigned int), st));
    void *args[] = {&a};
    EMS_CUDA(c, cudaLaunchCooperativeKernel((void *)k_pcg_grid_mg<P>, dim3(c->mg_blocks), dim3(512), args, 0, st));
    ++c->launches;
    return EMS_OK;
}

ems_status mg_solve(ems_ctx *c) {
    return c->prm.precision == EMS_F32 ? mg_solve_t<float>(c) : mg_solve_t<double>(c);
}

}  // namespace ems
