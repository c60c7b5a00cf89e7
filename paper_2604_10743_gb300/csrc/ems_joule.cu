// ems_joule.cu -- Joule-heating temperature profile along every branch
// (Sec. III-A: stationary thermal equation, thermal characteristic length,
// per-tree endpoint temperatures).
//
// Per segment s of thickness H_s: Gamma^2 = H_s t_ILD k_cu / k_ILD and the
// Joule rise Tm_s = j_s^2 rho Gamma^2 / k_cu.  With end temperatures T1 (the
// segment's a end, x = -L/2) and T2 (its b end) the stationary equation
// k T'' + j^2 rho - k (T - T0) / Gamma^2 = 0 gives
//   T(x) = T0 + Tm + (Tbar - T0 - Tm) cosh(x/G)/cosh(h) - Tn sinh(x/G)/sinh(h),
//   h = L / (2 G), Tbar = (T1 + T2)/2, Tn = (T1 - T2)/2,
// the physically consistent form of the printed solution (whose cos / sin
// terms solve the equation with the opposite sign of the loss term).
// IR nodes that are vias between layers, and pads, take the thermal map's
// value (T0 without a map); the other IR nodes carry zero net heat flow,
//   sum over incident segments of w (T_u coth 2h - T_v csch 2h - (T0 + Tm) tanh h) = 0,
// w = k_cu W H / G: a symmetric, diagonally dominant system along each tree
// (tridiagonal along a chain) eliminated leaf-to-root by one thread per tree.
#include <cmath>

#include "ems_internal.cuh"

namespace ems {
namespace {

struct JouleArgs {
    int n_trees, n_seg;
    int64_t N;
    double T0, rho, k_cu, k_ild, t_ild;
    const int64_t *toff;
    const int32_t *par, *face_seg, *child_ptr, *child_idx, *ir_id, *ir_par, *seg_a, *seg_b;
    const int8_t *fixed;
    const double *seg_L, *seg_H, *seg_W, *j, *node_x, *node_y, *nx, *ny, *raster;
    int rnx, rny;
    double rx0, ry0, rx1, ry1;
    double *T_ir, *Tn, *dg, *rb;       // dg, rb: [N] elimination scratch
};

struct SegTh { double G, Tm, w, cth, csh, th; };

__device__ __forceinline__ SegTh seg_thermal(const JouleArgs &a, int s) {
    SegTh q;
    q.G = sqrt(a.seg_H[s] * a.t_ild * a.k_cu / a.k_ild);
    q.Tm = a.j[s] * a.j[s] * a.rho * q.G * q.G / a.k_cu;
    q.w = a.k_cu * a.seg_W[s] * a.seg_H[s] / q.G;
    const double h = a.seg_L[s] / (2.0 * q.G);
    q.cth = 1.0 / tanh(2.0 * h);
    q.csh = 1.0 / sinh(2.0 * h);
    q.th = tanh(h);
    return q;
}

// the map's value at an IR node (bilinear over the vertex-centred raster,
// clamped at the border), or T0 without a map
__device__ double map_T(const JouleArgs &a, int u) {
    if (a.rnx == 0) return a.T0;
    double fx = (a.node_x[u] - a.rx0) / (a.rx1 - a.rx0) * (a.rnx - 1);
    double fy = (a.node_y[u] - a.ry0) / (a.ry1 - a.ry0) * (a.rny - 1);
    fx = fmin(fmax(fx, 0.0), (double)(a.rnx - 1));
    fy = fmin(fmax(fy, 0.0), (double)(a.rny - 1));
    const int ix = min((int)floor(fx), a.rnx - 2), iy = min((int)floor(fy), a.rny - 2);
    const double tx = fx - ix, ty = fy - iy;
    const double *r0 = a.raster + (int64_t)iy * a.rnx, *r1 = r0 + a.rnx;
    return (1 - tx) * (1 - ty) * r0[ix] + tx * (1 - ty) * r0[ix + 1] + (1 - tx) * ty * r1[ix] +
           tx * ty * r1[ix + 1];
}

// one thread per tree: temperatures of the tree's IR nodes
__global__ void k_joule_ir(JouleArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_trees) return;
    const int64_t cb = a.toff[t], n = a.toff[t + 1] - cb;
    // diagonal and right-hand side of every unconstrained IR node
    for (int64_t i = 0; i < n; ++i) {
        const int u = a.ir_id[cb + i];
        if (u < 0) continue;
        if (a.fixed[u]) { a.T_ir[u] = map_T(a, u); continue; }
        double d = 0.0, b = 0.0;
        auto seg = [&](int s) {
            const SegTh q = seg_thermal(a, s);
            d += q.w * q.cth;
            b += q.w * (a.T0 + q.Tm) * q.th;
            const int v = a.seg_a[s] + a.seg_b[s] - u;
            if (a.fixed[v]) b += q.w * q.csh * map_T(a, v);
        };
        if (i > 0) seg(a.face_seg[cb + i]);
        for (int k = a.child_ptr[cb + i]; k < a.child_ptr[cb + i + 1]; ++k) seg(a.face_seg[a.child_idx[k]]);
        a.dg[cb + i] = d;
        a.rb[cb + i] = b;
    }
    // leaf-to-root elimination into unconstrained parents
    for (int64_t i = n - 1; i >= 1; --i) {
        const int u = a.ir_id[cb + i];
        if (u < 0 || a.fixed[u]) continue;
        const int pl = a.ir_par[cb + i];
        const int P = a.ir_id[cb + pl];
        if (a.fixed[P]) continue;
        const SegTh q = seg_thermal(a, a.face_seg[cb + i]);
        const double off = q.w * q.csh;
        a.dg[cb + pl] -= off * off / a.dg[cb + i];
        a.rb[cb + pl] += off * a.rb[cb + i] / a.dg[cb + i];
    }
    // root-to-leaf substitution
    for (int64_t i = 0; i < n; ++i) {
        const int u = a.ir_id[cb + i];
        if (u < 0 || a.fixed[u]) continue;
        double b = a.rb[cb + i];
        if (i > 0) {
            const int P = a.ir_id[cb + a.ir_par[cb + i]];
            if (!a.fixed[P]) {
                const SegTh q = seg_thermal(a, a.face_seg[cb + i]);
                b += q.w * q.csh * a.T_ir[P];
            }
        }
        a.T_ir[u] = b / a.dg[cb + i];
    }
}

// per stress node: an IR node's temperature, or its segment's profile
__global__ void k_joule_profile(JouleArgs a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = a.ir_id[i];
        if (u >= 0) { a.Tn[i] = a.T_ir[u]; continue; }
        const int s = a.face_seg[i];
        const int ea = a.seg_a[s], eb = a.seg_b[s];
        const double frac = hypot(a.nx[i] - a.node_x[ea], a.ny[i] - a.node_y[ea]) /
                            hypot(a.node_x[eb] - a.node_x[ea], a.node_y[eb] - a.node_y[ea]);
        const double L = a.seg_L[s], x = (frac - 0.5) * L;
        const SegTh q = seg_thermal(a, s);
        const double h = L / (2.0 * q.G);
        const double T1 = a.T_ir[ea], T2 = a.T_ir[eb];
        const double Tbar = 0.5 * (T1 + T2), Tdn = 0.5 * (T1 - T2);
        a.Tn[i] = a.T0 + q.Tm + (Tbar - a.T0 - q.Tm) * cosh(x / q.G) / cosh(h) - Tdn * sinh(x / q.G) / sinh(h);
    }
}

}  // namespace
}  // namespace ems

using namespace ems;

extern "C" ems_status ems_joule_profile(ems_ctx *c, double k_cu, double k_ild, double t_ild) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "Joule profile before the first IR solve (it needs the currents)");
    if (!(k_cu > 0.0) || !(k_ild > 0.0) || !(t_ild > 0.0) || !std::isfinite(k_cu + k_ild + t_ild))
        return fail(c, EMS_E_INVAL, "k_cu, k_ild and t_ild must be positive and finite");
    Dev &d = c->d_all;
    JouleArgs a;
    a.n_trees = c->n_trees; a.n_seg = c->n_seg; a.N = c->N;
    a.T0 = c->prm.T0; a.rho = c->prm.rho_Cu; a.k_cu = k_cu; a.k_ild = k_ild; a.t_ild = t_ild;
    a.toff = d.toff; a.par = d.par; a.face_seg = d.face_seg; a.child_ptr = d.child_ptr; a.child_idx = d.child_idx;
    a.ir_id = d.ir_id; a.ir_par = d.ir_par; a.seg_a = d.seg_a; a.seg_b = d.seg_b; a.fixed = d.ir_fixed;
    a.seg_L = d.seg_L; a.seg_H = d.seg_H; a.seg_W = d.seg_W; a.j = d.j;      // sample 0's currents
    a.node_x = d.node_x; a.node_y = d.node_y; a.nx = d.nx_; a.ny = d.ny_; a.raster = d.raster;
    a.rnx = c->rnx; a.rny = c->rny; a.rx0 = c->rx0; a.ry0 = c->ry0; a.rx1 = c->rx1; a.ry1 = c->ry1;
    a.T_ir = d.T_ir; a.Tn = d.Tn; a.dg = d.sig_ss; a.rb = d.f;              // per-node scratch
    cudaStream_t st = c->stream;
    k_joule_ir<<<(c->n_trees + 127) / 128, 128, 0, st>>>(a);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    const int64_t blocks = std::min<int64_t>((c->N + 255) / 256, 8192);
    k_joule_profile<<<(unsigned)blocks, 256, 0, st>>>(a);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    c->joule = true;
    EMS_TRY(face_base(c));
    // kappa and the thermomigration term from the new temperatures (every
    // sample of the full layout; the first window with windows, the others
    // are rebuilt before use)
    if (windowed(c)) {
        map_window(c, 0, c->W);
        ems_status s = sample_physics(c);
        map_all(c);
        EMS_TRY(s);
    } else {
        EMS_TRY(sample_physics(c));
    }
    EMS_CUDA(c, cudaStreamSynchronize(st));
    return check_status(c);
}

extern "C" ems_status ems_get_node_temperature(ems_ctx *c, double *T) {
    if (!c || !T) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    EMS_CUDA(c, cudaMemcpyAsync(T, c->d.Tn, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}
