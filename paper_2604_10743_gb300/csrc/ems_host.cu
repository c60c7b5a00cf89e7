// ems_host.cu -- context, grid loading (tree extraction, packing, IR
// structure), workspace layout, state I/O of the GB300 EM/TM engine.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "ems_internal.cuh"
#include "../../include/ems_surrogate.h"

namespace ems {

ems_status fail(ems_ctx *c, ems_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

// Point the per-sample state arrays at samples [s0, s0 + ns); the per-node
// coefficient arrays, currents and IR work vectors (window-sized) keep their
// base: index 0 of a kernel's sample dimension is sample s0.
void map_window(ems_ctx *c, int s0, int ns) {
    Dev &d = c->d;
    d = c->d_all;
    const size_t nt = (size_t)c->n_trees, ns_ = (size_t)c->n_seg, nv = nt * (size_t)c->maxv;
    auto off = [&](auto *&ptr, size_t stride) {
        if (ptr) ptr += (size_t)s0 * stride;
    };
    off(d.R, ns_); off(d.j, ns_); off(d.R_prev, ns_); off(d.kfac, ns_); off(d.sfac, ns_);
    off(d.u, (size_t)c->n_nodes);
    off(d.drop, 1); off(d.ir_iters, 1); off(d.gttf, 1); off(d.gdrops, (size_t)c->prm.n_outer + 1);
    d.sig = (char *)d.sig + (size_t)s0 * (size_t)c->P * elem_bytes(c);
    off(d.v_count, nt); off(d.dirty, nt); off(d.mortal, nt); off(d.ssmax, nt);
    off(d.kr_mode, nt); off(d.kdone, nt); off(d.sched, nt); off(d.fdt, nt);
    off(d.v_node, nv); off(d.v_seg, nv); off(d.v_vol, nv); off(d.v_tnuc, nv);
    off(d.feat, nt * EMS_MLP_FEATURES); off(d.pred, nt * EMS_MLP_OUTPUTS);
    off(d.pert, (size_t)EMS_MAX_PERT);
    c->S = ns;
    c->win_s0 = s0;
}

void map_all(ems_ctx *c) {
    c->d = c->d_all;
    c->S = c->S_all;
    c->win_s0 = 0;
}

ems_status cuda_check(ems_ctx *c, cudaError_t e, const char *what) {
    cudaGetLastError();   // clear the error slot so later calls do not report it again
    return fail(c, EMS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t elem_bytes(const ems_ctx *c) { return c->prm.precision == EMS_F32 ? 4 : 8; }

namespace {

// ---------------------------------------------------------------------------
// Input validation
// ---------------------------------------------------------------------------
bool finite_pos(const double *a, int n) {
    for (int i = 0; i < n; ++i)
        if (!(std::isfinite(a[i]) && a[i] > 0.0)) return false;
    return true;
}

ems_status validate(ems_ctx *c, const ems_params *p, const ems_grid_desc *g) {
    if (!p || !g) return fail(c, EMS_E_INVAL, "null params or grid");
    if (g->n_nodes <= 0 || g->n_seg <= 0 || g->n_pads <= 0)
        return fail(c, EMS_E_INVAL, "grid needs nodes, segments and at least one pad");
    if (!g->node_x || !g->node_y || !g->seg_a || !g->seg_b || !g->seg_layer || !g->seg_cells ||
        !g->seg_R0 || !g->seg_W || !g->seg_H || !g->seg_L || !g->pad_node || !g->pad_V)
        return fail(c, EMS_E_INVAL, "null grid array");
    if (g->n_sinks > 0 && (!g->sink_node || !g->sink_I))
        return fail(c, EMS_E_INVAL, "null sink array");
    for (int i = 0; i < g->n_nodes; ++i)
        if (!std::isfinite(g->node_x[i]) || !std::isfinite(g->node_y[i]))
            return fail(c, EMS_E_INVAL, "non-finite node coordinate");
    for (int s = 0; s < g->n_seg; ++s) {
        if (g->seg_a[s] < 0 || g->seg_a[s] >= g->n_nodes || g->seg_b[s] < 0 ||
            g->seg_b[s] >= g->n_nodes || g->seg_a[s] == g->seg_b[s])
            return fail(c, EMS_E_INVAL, "segment end out of range");
        if (g->seg_cells[s] < 1) return fail(c, EMS_E_INVAL, "segment with < 1 FD cell");
    }
    if (g->seg_via)
        for (int s = 0; s < g->n_seg; ++s)
            if (g->seg_via[s] != 0 && g->seg_via[s] != 1) return fail(c, EMS_E_INVAL, "seg_via must be 0 or 1");
    if (!finite_pos(g->seg_R0, g->n_seg) || !finite_pos(g->seg_W, g->n_seg) ||
        !finite_pos(g->seg_H, g->n_seg) || !finite_pos(g->seg_L, g->n_seg))
        return fail(c, EMS_E_INVAL, "non-positive or non-finite segment R, W, H or L");
    for (int i = 0; i < g->n_pads; ++i)
        if (g->pad_node[i] < 0 || g->pad_node[i] >= g->n_nodes || !std::isfinite(g->pad_V[i]))
            return fail(c, EMS_E_INVAL, "bad pad");
    for (int i = 0; i < g->n_sinks; ++i)
        if (g->sink_node[i] < 0 || g->sink_node[i] >= g->n_nodes || !std::isfinite(g->sink_I[i]))
            return fail(c, EMS_E_INVAL, "bad sink (index or NaN current)");
    int S = g->n_samples > 0 ? g->n_samples : 1;
    if ((g->kappa_factor || g->sigc_factor) && g->n_samples <= 0)
        return fail(c, EMS_E_INVAL, "MC factors need n_samples > 0");
    for (const double *fct : {g->kappa_factor, g->sigc_factor})
        if (fct && !finite_pos(fct, S * g->n_seg))
            return fail(c, EMS_E_INVAL, "non-positive MC factor");
    if (!(p->sigma_crit > 0.0) || !(p->delta > 0.0) || !(p->B_modulus > 0.0) ||
        !(p->T0 > 0.0) || !(p->D0 > 0.0) || p->n_inner < 1 || p->n_outer < 1 ||
        !(p->horizon > 0.0) || p->max_voids_per_tree < 1 ||
        p->max_voids_per_tree > EMS_MAX_VOIDS || p->ir_max_iter < 1 || !(p->ir_rtol > 0.0) ||
        (p->ir_precond != EMS_PC_AUTO && p->ir_precond != EMS_PC_JACOBI))
        return fail(c, EMS_E_INVAL, "bad parameter value");
    if (p->precision != EMS_F64 && p->precision != EMS_F32)
        return fail(c, EMS_E_INVAL, "precision must be EMS_F64 or EMS_F32");
    if (p->method != EMS_BE && p->method != EMS_KRYLOV && p->method != EMS_AUTO)
        return fail(c, EMS_E_INVAL, "method must be EMS_BE, EMS_KRYLOV or EMS_AUTO");
    if (p->method != EMS_BE && (p->krylov_q < 1 || p->krylov_q > 40 || !(p->krylov_eta > 0.0)))
        return fail(c, EMS_E_INVAL, "krylov_q must be 1..40 and krylov_eta > 0");
    if (p->window_samples < 0) return fail(c, EMS_E_INVAL, "window_samples must be >= 0");
    if (!(p->krylov_eps >= 0.0 && p->krylov_eps < 1.0)) return fail(c, EMS_E_INVAL, "krylov_eps must be in [0, 1)");
    if (p->window_samples > 0 && p->window_samples < S && p->method != EMS_BE)
        return fail(c, EMS_E_INVAL, "the reduced models need every sample's coefficients: window_samples 0");
    return EMS_OK;
}

// Every node must reach a pad through segments (else the IR system is singular).
bool connected_to_pads(const ems_grid_desc *g) {
    int n = g->n_nodes;
    std::vector<int> deg(n + 1, 0);
    for (int s = 0; s < g->n_seg; ++s) { deg[g->seg_a[s] + 1]++; deg[g->seg_b[s] + 1]++; }
    for (int i = 0; i < n; ++i) deg[i + 1] += deg[i];
    std::vector<int> adj(deg[n]), pos(deg.begin(), deg.end() - 1);
    for (int s = 0; s < g->n_seg; ++s) {
        adj[pos[g->seg_a[s]]++] = g->seg_b[s];
        adj[pos[g->seg_b[s]]++] = g->seg_a[s];
    }
    std::vector<uint8_t> seen(n, 0);
    std::vector<int> st;
    for (int i = 0; i < g->n_pads; ++i)
        if (!seen[g->pad_node[i]]) { seen[g->pad_node[i]] = 1; st.push_back(g->pad_node[i]); }
    while (!st.empty()) {
        int u = st.back(); st.pop_back();
        for (int k = deg[u]; k < deg[u + 1]; ++k)
            if (!seen[adj[k]]) { seen[adj[k]] = 1; st.push_back(adj[k]); }
    }
    for (int i = 0; i < n; ++i)
        if (!seen[i]) return false;
    return true;
}

int find(std::vector<int> &p, int x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

// ---------------------------------------------------------------------------
// Tree extraction in canonical order (see ems.h)
// ---------------------------------------------------------------------------
ems_status extract_trees(ems_ctx *c, const ems_grid_desc *g, HostTrees &tr) {
    const int ns = g->n_seg;
    auto is_via = [&](int s) { return g->seg_via && g->seg_via[s]; };
    // (layer, node) groups of incident wire segments, in (layer, node,
    // segment) order by a counting sort of the endpoint records into per-layer
    // node buckets (via resistors join layers and belong to no stress tree)
    const int nn_ = g->n_nodes;
    int lay_idx[65];
    std::fill(lay_idx, lay_idx + 65, -1);
    for (int s = 0; s < ns; ++s)
        if (!is_via(s)) lay_idx[g->seg_layer[s]] = 0;
    int nL = 0;
    for (int l = 0; l < 65; ++l)
        if (lay_idx[l] == 0) lay_idx[l] = nL++;
    const int64_t nb = (int64_t)nL * nn_;
    std::vector<int64_t> bstart(nb + 1, 0);
    for (int s = 0; s < ns; ++s) {
        if (is_via(s)) continue;
        const int64_t li = lay_idx[g->seg_layer[s]];
        ++bstart[li * nn_ + g->seg_a[s] + 1];
        ++bstart[li * nn_ + g->seg_b[s] + 1];
    }
    for (int64_t k = 0; k < nb; ++k) bstart[k + 1] += bstart[k];
    struct Rec { int32_t layer, node, seg; };
    std::vector<Rec> rec((size_t)bstart[nb]);
    {
        std::vector<int64_t> fill(bstart.begin(), bstart.end() - 1);
        for (int s = 0; s < ns; ++s) {
            if (is_via(s)) continue;
            const int64_t li = lay_idx[g->seg_layer[s]];
            rec[fill[li * nn_ + g->seg_a[s]]++] = {g->seg_layer[s], g->seg_a[s], s};
            rec[fill[li * nn_ + g->seg_b[s]]++] = {g->seg_layer[s], g->seg_b[s], s};
        }
    }
    std::vector<int64_t> gstart;          // group boundaries in rec
    std::vector<int32_t> grp_of((size_t)nb, -1);   // bucket (layer index, node) -> group
    for (int64_t k = 0; k < nb; ++k)
        if (bstart[k + 1] > bstart[k]) {
            grp_of[k] = (int32_t)gstart.size();
            gstart.push_back(bstart[k]);
        }
    gstart.push_back((int64_t)rec.size());
    const size_t ng = gstart.size() - 1;
    std::vector<int> uf(ns);
    std::iota(uf.begin(), uf.end(), 0);
    for (size_t q = 0; q < ng; ++q)
        for (int64_t k = gstart[q] + 1; k < gstart[q + 1]; ++k) {
            int a = find(uf, rec[gstart[q]].seg), b = find(uf, rec[k].seg);
            if (a != b) uf[std::max(a, b)] = std::min(a, b);
        }
    // tree ids in order of smallest segment id
    std::vector<int32_t> tid_of_root(ns, -1);
    tr.tree_of_seg.assign(ns, -1);
    std::vector<std::vector<int32_t>> tsegs;
    for (int s = 0; s < ns; ++s) {
        if (is_via(s)) continue;
        int r = find(uf, s);
        if (tid_of_root[r] < 0) { tid_of_root[r] = (int32_t)tsegs.size(); tsegs.emplace_back(); }
        tr.tree_of_seg[s] = tid_of_root[r];
        tsegs[tid_of_root[r]].push_back(s);
    }
    tr.n_trees = (int)tsegs.size();
    auto group_of = [&](int32_t layer, int32_t node) -> int32_t {
        const int li = layer >= 0 && layer < 65 ? lay_idx[layer] : -1;
        return li < 0 ? -1 : grp_of[(size_t)li * nn_ + node];
    };
    // pass 1, per tree (in parallel): root (lowest-id leaf), stress nodes
    // (root + every segment's cells) and incidence entries (an IR node lists
    // its group's segments, an interior node its own segment)
    const int nt = tr.n_trees;
    std::vector<int32_t> root_of(nt, -1);
    std::vector<int64_t> nn(nt, 0), ni(nt, 0);
    std::vector<int> bad(nt, 0);            // 1: a cycle, 2: no leaf
    parallel_for(nt, [&](int t) {
        const auto &ts = tsegs[t];
        const int32_t layer = g->seg_layer[ts[0]];
        std::vector<int32_t> nodes;
        nodes.reserve(2 * ts.size());
        for (int s : ts) { nodes.push_back(g->seg_a[s]); nodes.push_back(g->seg_b[s]); }
        std::sort(nodes.begin(), nodes.end());
        nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
        if (nodes.size() != ts.size() + 1) { bad[t] = 1; return; }
        int64_t cnt = 1, inc = 0;
        for (int32_t nd : nodes) {
            const int32_t q = group_of(layer, nd);
            const int64_t gs = gstart[q + 1] - gstart[q];
            inc += gs;
            if (root_of[t] < 0 && gs == 1) root_of[t] = nd;      // nodes sorted: lowest id
        }
        if (root_of[t] < 0) { bad[t] = 2; return; }
        for (int s : ts) { cnt += g->seg_cells[s]; inc += g->seg_cells[s] - 1; }
        nn[t] = cnt;
        ni[t] = inc;
    });
    for (int t = 0; t < nt; ++t) {
        if (bad[t] == 1) return fail(c, EMS_E_INVAL, "same-layer component with a cycle: not a tree");
        if (bad[t] == 2) return fail(c, EMS_E_INVAL, "tree without a leaf");
    }
    tr.off.assign(nt + 1, 0);
    std::vector<int64_t> ioff(nt + 1, 0);
    for (int t = 0; t < nt; ++t) { tr.off[t + 1] = tr.off[t] + nn[t]; ioff[t + 1] = ioff[t] + ni[t]; }
    const int64_t total = tr.off[nt];
    tr.par.resize(total); tr.face_seg.resize(total); tr.face_dx.resize(total);
    tr.face_area.resize(total); tr.face_sign.resize(total); tr.x.resize(total);
    tr.y.resize(total); tr.owner_seg.resize(total); tr.ir_id.resize(total); tr.ir_par.resize(total);
    tr.inc_ptr.assign(total + 1, 0);
    tr.inc_seg.resize(ioff[nt]);
    tr.is_chain.assign(nt, 1);

    // pass 2, per tree (in parallel): depth-first preorder from the root into
    // the tree's own range, the canonical order
    parallel_for(nt, [&](int t) {
        const auto &ts = tsegs[t];
        const int32_t layer = g->seg_layer[ts[0]];
        const int32_t root = root_of[t];
        const int64_t base = tr.off[t];
        int64_t ip = ioff[t];
        int32_t cnt = 0;
        auto emit = [&](int32_t parent, int32_t seg, double dx, double area, int8_t sign, double xx,
                        double yy, int32_t own, int32_t grp, int32_t irn, int32_t irp) -> int32_t {
            const int64_t i = base + cnt;
            tr.ir_id[i] = irn; tr.ir_par[i] = irp;
            tr.par[i] = parent; tr.face_seg[i] = seg; tr.face_dx[i] = dx;
            tr.face_area[i] = area; tr.face_sign[i] = sign;
            tr.x[i] = xx; tr.y[i] = yy; tr.owner_seg[i] = own;
            if (grp >= 0) {
                for (int64_t k = gstart[grp]; k < gstart[grp + 1]; ++k) tr.inc_seg[ip++] = rec[k].seg;
            } else {
                tr.inc_seg[ip++] = seg;
            }
            tr.inc_ptr[i + 1] = (int32_t)ip;
            return cnt++;
        };
        int32_t rg = group_of(layer, root);
        emit(-1, -1, 0.0, 0.0, 0, g->node_x[root], g->node_y[root], rec[gstart[rg]].seg, rg, root, -1);
        // depth-first preorder: ("node", ir, local, came) or ("seg", pir, plocal, seg, cir)
        struct Item { int kind; int32_t u, lu, s, w; };
        std::vector<Item> stack;
        stack.push_back({0, root, 0, -1, -1});
        std::vector<int32_t> kids;
        while (!stack.empty()) {
            Item it = stack.back(); stack.pop_back();
            if (it.kind == 0) {
                int32_t q = group_of(layer, it.u);
                kids.clear();
                for (int64_t k = gstart[q]; k < gstart[q + 1]; ++k)
                    if (rec[k].seg != it.s) kids.push_back(rec[k].seg);
                for (auto k = kids.rbegin(); k != kids.rend(); ++k) {
                    int32_t s = *k;
                    int32_t w = g->seg_a[s] == it.u ? g->seg_b[s] : g->seg_a[s];
                    stack.push_back({1, it.u, it.lu, s, w});
                }
            } else {
                const int32_t s = it.s, u = it.u, w = it.w;
                const int cells = g->seg_cells[s];
                const double dx = g->seg_L[s] / cells, area = g->seg_W[s] * g->seg_H[s];
                const int8_t sign = g->seg_a[s] == u ? 1 : -1;
                int32_t prev = it.lu;
                for (int k = 1; k < cells; ++k) {
                    double f = (double)k / cells;
                    prev = emit(prev, s, dx, area, sign,
                                g->node_x[u] + f * (g->node_x[w] - g->node_x[u]),
                                g->node_y[u] + f * (g->node_y[w] - g->node_y[u]), s, -1, -1, -1);
                }
                int32_t wg = group_of(layer, w);
                int32_t lw = emit(prev, s, dx, area, sign, g->node_x[w], g->node_y[w],
                                  rec[gstart[wg]].seg, wg, w, it.lu);
                stack.push_back({0, w, lw, s, -1});
            }
        }
        for (int32_t i = 1; i < cnt; ++i)
            if (tr.par[base + i] != i - 1) { tr.is_chain[t] = 0; break; }
    });
    // children CSR (tree-local indices)
    const int64_t N = tr.off.back();
    tr.child_ptr.assign(N + 1, 0);
    for (int t = 0; t < tr.n_trees; ++t)
        for (int64_t i = tr.off[t] + 1; i < tr.off[t + 1]; ++i) tr.child_ptr[tr.off[t] + tr.par[i] + 1]++;
    for (int64_t i = 0; i < N; ++i) tr.child_ptr[i + 1] += tr.child_ptr[i];
    tr.child_idx.assign(tr.child_ptr[N], 0);
    std::vector<int32_t> fill(tr.child_ptr.begin(), tr.child_ptr.end() - 1);
    for (int t = 0; t < tr.n_trees; ++t)
        for (int64_t i = tr.off[t] + 1; i < tr.off[t + 1]; ++i)
            tr.child_idx[fill[tr.off[t] + tr.par[i]]++] = (int32_t)(i - tr.off[t]);
    return EMS_OK;
}

// IR structure on the free (non-pad) nodes
struct HostIR {
    std::vector<int32_t> free_of_node, node_of_free, ptr, col, ent_ptr, ent_seg, rhs_ptr, rhs_seg;
    std::vector<int8_t> ent_diag;
    std::vector<double> rhs_padV, sink;
    std::vector<double> padV_of_node;
};

void build_ir(const ems_grid_desc *g, HostIR &ir) {
    const int n = g->n_nodes;
    ir.padV_of_node.assign(n, NAN);
    for (int i = 0; i < g->n_pads; ++i) ir.padV_of_node[g->pad_node[i]] = g->pad_V[i];
    ir.free_of_node.assign(n, -1);
    for (int i = 0; i < n; ++i)
        if (std::isnan(ir.padV_of_node[i])) {
            ir.free_of_node[i] = (int32_t)ir.node_of_free.size();
            ir.node_of_free.push_back(i);
        }
    const int nf = (int)ir.node_of_free.size();
    // per free row its (col, seg, diag) contributions and its pad segments,
    // gathered by a counting sort over the segments (ascending segment id)
    struct E { int32_t col, seg; int8_t diag; };
    std::vector<int64_t> eoff((size_t)nf + 1, 0), poff((size_t)nf + 1, 0);
    for (int s = 0; s < g->n_seg; ++s) {
        const int fa = ir.free_of_node[g->seg_a[s]], fb = ir.free_of_node[g->seg_b[s]];
        if (fa >= 0) { eoff[fa + 1] += fb >= 0 ? 2 : 1; if (fb < 0) ++poff[fa + 1]; }
        if (fb >= 0) { eoff[fb + 1] += fa >= 0 ? 2 : 1; if (fa < 0) ++poff[fb + 1]; }
    }
    for (int r = 0; r < nf; ++r) { eoff[r + 1] += eoff[r]; poff[r + 1] += poff[r]; }
    std::vector<E> ent((size_t)eoff[nf]);
    ir.rhs_seg.resize((size_t)poff[nf]);
    ir.rhs_padV.resize((size_t)poff[nf]);
    {
        std::vector<int64_t> ep(eoff.begin(), eoff.end() - 1), pp(poff.begin(), poff.end() - 1);
        for (int s = 0; s < g->n_seg; ++s) {
            const int a = g->seg_a[s], b = g->seg_b[s];
            const int fa = ir.free_of_node[a], fb = ir.free_of_node[b];
            if (fa >= 0) {
                ent[ep[fa]++] = {fa, s, 1};
                if (fb >= 0) ent[ep[fa]++] = {fb, s, 0};
                else { ir.rhs_seg[pp[fa]] = s; ir.rhs_padV[pp[fa]++] = ir.padV_of_node[b]; }
            }
            if (fb >= 0) {
                ent[ep[fb]++] = {fb, s, 1};
                if (fa >= 0) ent[ep[fb]++] = {fa, s, 0};
                else { ir.rhs_seg[pp[fb]] = s; ir.rhs_padV[pp[fb]++] = ir.padV_of_node[a]; }
            }
        }
    }
    ir.rhs_ptr.resize((size_t)nf + 1);
    for (int r = 0; r <= nf; ++r) ir.rhs_ptr[r] = (int32_t)poff[r];
    // rows in parallel blocks: entries sorted by (col, seg), one matrix entry
    // per distinct column listing its segments
    const int nblk = std::max(1, std::min(1024, nf / 4096));
    std::vector<int32_t> ncol((size_t)nf);
    auto rows_of = [&](int q, int &r0, int &r1) {
        r0 = (int)((int64_t)nf * q / nblk); r1 = (int)((int64_t)nf * (q + 1) / nblk);
    };
    parallel_for(nblk, [&](int q) {
        int r0, r1;
        rows_of(q, r0, r1);
        for (int r = r0; r < r1; ++r) {
            E *v = ent.data() + eoff[r], *ve = ent.data() + eoff[r + 1];
            std::sort(v, ve, [](const E &x, const E &y) { return x.col != y.col ? x.col < y.col : x.seg < y.seg; });
            int32_t k = 0;
            for (E *e = v; e < ve; ++e)
                if (e == v || e->col != (e - 1)->col) ++k;
            ncol[r] = k;
        }
    });
    ir.ptr.resize((size_t)nf + 1);
    ir.ptr[0] = 0;
    for (int r = 0; r < nf; ++r) ir.ptr[r + 1] = ir.ptr[r] + ncol[r];
    const size_t nnz = (size_t)ir.ptr[nf];
    ir.col.resize(nnz);
    ir.ent_diag.resize(nnz);
    ir.ent_ptr.resize(nnz + 1);
    ir.ent_seg.resize((size_t)eoff[nf]);
    ir.ent_ptr[0] = 0;
    parallel_for(nblk, [&](int q) {
        int r0, r1;
        rows_of(q, r0, r1);
        for (int r = r0; r < r1; ++r) {
            int64_t j = (int64_t)ir.ptr[r] - 1;        // the current entry (column group)
            for (int64_t k = eoff[r]; k < eoff[r + 1]; ++k) {
                const E &e = ent[k];
                if (k == eoff[r] || e.col != ent[k - 1].col) {
                    if (k > eoff[r]) ir.ent_ptr[j + 1] = (int32_t)k;      // end of entry j
                    ++j;
                    ir.col[j] = e.col;
                    ir.ent_diag[j] = e.diag;
                }
                ir.ent_seg[k] = e.seg;
            }
            if (eoff[r + 1] > eoff[r]) ir.ent_ptr[j + 1] = (int32_t)eoff[r + 1];
        }
    });
    ir.sink.assign(nf, 0.0);
    for (int i = 0; i < g->n_sinks; ++i) {
        int f = ir.free_of_node[g->sink_node[i]];
        if (f >= 0) ir.sink[f] += g->sink_I[i];
    }
}

// ---------------------------------------------------------------------------
// Workspace layout: every device array carved from one block
// ---------------------------------------------------------------------------
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <class T> T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

struct Plan {
    HostTrees tr;
    HostIR ir;
    MGHost mg;
    std::vector<TreePack> pack;
    int64_t P = 0;
    int S = 1;      // samples whose state the context holds
    int Sd = 1;     // samples whose per-node coefficients and IR vectors it holds at once
};

ems_status make_plan(ems_ctx *c, const ems_params *p, const ems_grid_desc *g, Plan &pl) {
    EMS_TRY(validate(c, p, g));
    if (!connected_to_pads(g)) return fail(c, EMS_E_INVAL, "node not connected to any pad");
    EMS_TRY(extract_trees(c, g, pl.tr));
    build_ir(g, pl.ir);
    if (p->ir_precond == EMS_PC_AUTO)
        mg_build((int)pl.ir.node_of_free.size(), pl.ir.ptr, pl.ir.col, pl.ir.ent_ptr, pl.ir.ent_seg,
                 pl.ir.ent_diag, g->seg_R0, 1024, pl.mg);
    pl.S = g->n_samples > 0 ? g->n_samples : 1;
    pl.Sd = (p->window_samples > 0 && p->window_samples < pl.S) ? p->window_samples : pl.S;
    pl.pack.resize(pl.tr.n_trees);
    int64_t P = 0;
    for (int t = 0; t < pl.tr.n_trees; ++t) {
        int64_t n = pl.tr.off[t + 1] - pl.tr.off[t];
        int T = 0, M = 0, CL = 1;
        int kind = 0;
        if (pl.tr.is_chain[t]) chain_shape(n, p->precision, p->method, c ? &c->rules : nullptr, &T, &M, &CL, &kind);
        TreePack tp;
        if (T > 0) { tp.T = T; tp.M = M; tp.CL = CL; tp.kind = kind; tp.pbase = P; P += (int64_t)T * M; }
        else { tp.T = 1; tp.M = (int)n; tp.pbase = P; P += (n + 31) / 32 * 32; }
        pl.pack[t] = tp;
    }
    pl.P = P;
    return EMS_OK;
}

// One-slot cache of the last plan ems_workspace_bytes made, so that the
// usual sequence (size query, workspace allocation, ems_load_grid) plans once.
// The key hashes everything planning reads: the parameters it depends on, the shape rules,
// the grid's sizes and the arrays of its topology, geometry, pads, sinks and
// initial resistances (not the Monte Carlo factors or the map: validate()
// checks those on every load).
struct PlanCache {
    std::mutex mu;
    bool valid = false;
    uint64_t key = 0;
    Plan plan;
};
PlanCache &plan_cache() {
    static PlanCache pc;
    return pc;
}

struct Hasher {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    void mix(uint64_t v) {
        h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 31;
    }
    void bytes(const void *p, size_t n) {
        mix(n);
        if (!p) { mix(0xFFFFFFFFull); return; }
        const unsigned char *b = (const unsigned char *)p;
        size_t k = 0;
        for (; k + 8 <= n; k += 8) {
            uint64_t v;
            std::memcpy(&v, b + k, 8);
            mix(v);
        }
        uint64_t t = 0;
        for (; k < n; ++k) t = (t << 8) | b[k];
        mix(t);
    }
};

uint64_t plan_key(const ems_params *p, const std::vector<ems_chain_rule> &rules, const ems_grid_desc *g) {
    Hasher h;
    // the parameters the plan depends on (field by field: the struct has padding)
    h.mix((uint64_t)(int64_t)p->precision); h.mix((uint64_t)(int64_t)p->method);
    h.mix((uint64_t)(int64_t)p->ir_precond); h.mix((uint64_t)(int64_t)p->window_samples);
    h.bytes(rules.data(), rules.size() * sizeof(ems_chain_rule));
    const size_t nn = g->n_nodes > 0 ? (size_t)g->n_nodes : 0, ns = g->n_seg > 0 ? (size_t)g->n_seg : 0;
    const size_t np = g->n_pads > 0 ? (size_t)g->n_pads : 0, nk = g->n_sinks > 0 ? (size_t)g->n_sinks : 0;
    h.mix(nn); h.mix(ns); h.mix(np); h.mix(nk); h.mix((uint64_t)(int64_t)g->n_samples);
    h.bytes(g->node_x, 8 * nn); h.bytes(g->node_y, 8 * nn);
    h.bytes(g->seg_a, 4 * ns); h.bytes(g->seg_b, 4 * ns); h.bytes(g->seg_layer, 4 * ns);
    h.bytes(g->seg_cells, 4 * ns); h.bytes(g->seg_R0, 8 * ns); h.bytes(g->seg_W, 8 * ns);
    h.bytes(g->seg_H, 8 * ns); h.bytes(g->seg_L, 8 * ns); h.bytes(g->seg_via, ns);
    h.bytes(g->pad_node, 4 * np); h.bytes(g->pad_V, 8 * np);
    h.bytes(g->sink_node, 4 * nk); h.bytes(g->sink_I, 8 * nk);
    return h.h;
}

size_t carve(ems_ctx *c, const Plan &pl, const ems_grid_desc *g, void *base, Dev &d) {
    Carver cv(base);
    // per-sample state: S samples; per-node coefficients, currents and IR
    // work vectors: Sd samples (a window, or all of them)
    const int S = pl.S, Sd = pl.Sd, ns = g->n_seg, nn = g->n_nodes, nf = (int)pl.ir.node_of_free.size();
    const int64_t nnz = (int64_t)pl.ir.col.size(), N = pl.tr.off.back(), P = pl.P;
    const int nt = pl.tr.n_trees;
    const int maxv = c ? c->prm.max_voids_per_tree : EMS_MAX_VOIDS;
    const size_t eb = (c && c->prm.precision == EMS_F32) ? 4 : 8;
    d.seg_a = cv.take<int32_t>(ns); d.seg_b = cv.take<int32_t>(ns);
    d.seg_R0 = cv.take<double>(ns); d.seg_W = cv.take<double>(ns); d.seg_H = cv.take<double>(ns);
    d.R = cv.take<double>((size_t)S * ns); d.j = cv.take<double>((size_t)S * ns);
    d.ir_free_of_node = cv.take<int32_t>(nn); d.ir_node_of_free = cv.take<int32_t>(nf);
    d.csr_ptr = cv.take<int32_t>(nf + 1); d.csr_col = cv.take<int32_t>(nnz);
    d.ent_ptr = cv.take<int32_t>(nnz + 1); d.ent_seg = cv.take<int32_t>(pl.ir.ent_seg.size());
    d.ent_diag = cv.take<int8_t>(nnz);
    d.rhs_ptr = cv.take<int32_t>(nf + 1); d.rhs_seg = cv.take<int32_t>(pl.ir.rhs_seg.size() + 1);
    d.rhs_padV = cv.take<double>(pl.ir.rhs_padV.size() + 1);
    d.sink_of_free = cv.take<double>(nf);
    d.csr_val = cv.take<double>((size_t)Sd * nnz);
    d.ir_b = cv.take<double>((size_t)Sd * nf); d.ir_dinv = cv.take<double>((size_t)Sd * nf);
    d.ir_x = cv.take<double>((size_t)Sd * nf); d.ir_r = cv.take<double>((size_t)Sd * nf);
    d.ir_p = cv.take<double>((size_t)Sd * nf); d.ir_Ap = cv.take<double>((size_t)Sd * nf);
    d.ir_z = cv.take<double>((size_t)Sd * nf);
    d.val32 = cv.take<float>((size_t)Sd * nnz); d.dinv32 = cv.take<float>((size_t)Sd * nf);
    d.r32 = cv.take<float>((size_t)Sd * nf); d.p32 = cv.take<float>((size_t)Sd * nf);
    d.Ap32 = cv.take<float>((size_t)Sd * nf); d.z32 = cv.take<float>((size_t)Sd * nf);
    d.d32 = cv.take<float>((size_t)Sd * nf);
    d.u = cv.take<double>((size_t)S * nn); d.pad_V_of_node = cv.take<double>(nn);
    d.drop = cv.take<double>(S);
    d.red = cv.take<double>(4096 + 8 * (size_t)S);
    d.ir_iters = cv.take<int32_t>(S);
    d.gbar = cv.take<unsigned int>(64);
    d.toff = cv.take<int64_t>(nt + 1);
    d.par = cv.take<int32_t>(N); d.face_seg = cv.take<int32_t>(N); d.owner_seg = cv.take<int32_t>(N);
    d.inc_ptr = cv.take<int32_t>(N + 1); d.inc_seg = cv.take<int32_t>(pl.tr.inc_seg.size());
    d.child_ptr = cv.take<int32_t>(N + 1); d.child_idx = cv.take<int32_t>(pl.tr.child_idx.size() + 1);
    d.face_sign = cv.take<int8_t>(N);
    d.face_dx = cv.take<double>(N); d.face_area = cv.take<double>(N);
    d.nx_ = cv.take<double>(N); d.ny_ = cv.take<double>(N);
    d.Tn = cv.take<double>(N); d.Mface = cv.take<double>((size_t)Sd * N); d.V = cv.take<double>(N);
    d.fb_ka = cv.take<double>(N); d.fb_g = cv.take<double>(N); d.fb_M = cv.take<double>(N);
    d.kap_a = cv.take<double>((size_t)Sd * N); d.g = cv.take<double>((size_t)Sd * N);
    d.leak = cv.take<double>((size_t)Sd * N); d.thr = cv.take<double>((size_t)Sd * N);
    d.f = cv.take<double>((size_t)Sd * N); d.sig_ss = cv.take<double>((size_t)Sd * N);
    d.pbase = cv.take<int64_t>(nt); d.pT = cv.take<int32_t>(nt); d.pM = cv.take<int32_t>(nt);
    d.sig = cv.take<char>((size_t)S * P * eb); d.alpha = cv.take<char>((size_t)Sd * P * eb);
    d.beta = cv.take<char>((size_t)Sd * P * eb); d.gam = cv.take<char>((size_t)Sd * P * eb);
    d.uu = cv.take<char>((size_t)Sd * P * eb); d.Pf = cv.take<char>((size_t)Sd * P * eb);
    d.Pb = cv.take<char>((size_t)Sd * P * eb); d.pinv = cv.take<double>((size_t)Sd * P);
    d.dtg = cv.take<char>((size_t)Sd * P * eb); d.dtl = cv.take<char>((size_t)Sd * P * eb);
    d.kc = cv.take<char>((size_t)Sd * P * eb);
    d.v_count = cv.take<int32_t>((size_t)S * nt);
    d.v_node = cv.take<int32_t>((size_t)S * nt * maxv); d.v_seg = cv.take<int32_t>((size_t)S * nt * maxv);
    d.v_vol = cv.take<double>((size_t)S * nt * maxv); d.v_tnuc = cv.take<double>((size_t)S * nt * maxv);
    d.dirty = cv.take<int32_t>((size_t)S * nt);
    d.status = cv.take<int32_t>(8); d.counters = cv.take<int32_t>(8);
    d.mortal = cv.take<uint8_t>((size_t)S * nt); d.ssmax = cv.take<double>((size_t)S * nt);
    d.kfac = cv.take<double>((size_t)S * ns); d.sfac = cv.take<double>((size_t)S * ns);
    d.thr0 = cv.take<double>((size_t)Sd * N);
    d.R_prev = cv.take<double>((size_t)S * ns);
    d.raster = cv.take<double>(EMS_MAX_RASTER);
    d.pert = cv.take<double>((size_t)S * EMS_MAX_PERT);
    d.kr_mode = cv.take<int32_t>((size_t)S * nt); d.kdone = cv.take<int32_t>((size_t)S * nt);
    {
        const int no = c ? c->prm.n_outer : 1;
        d.gtime = cv.take<double>(1); d.gttf = cv.take<double>(S);
        d.gdrops = cv.take<double>((size_t)S * (no + 1)); d.giters = cv.take<double>(1);
        d.gstep = cv.take<int32_t>(1);
    }
    d.feat = cv.take<float>((size_t)S * nt * EMS_MLP_FEATURES);
    d.pred = cv.take<float>((size_t)S * nt * EMS_MLP_OUTPUTS);
    d.mg_i = cv.take<int32_t>(pl.mg.ints.size() + 1);
    d.mg_d = cv.take<double>(pl.mg.dbls.size() + 1);
    d.mg_f = cv.take<float>(pl.mg.dbls.size() + 1);
    d.mg_sc = cv.take<double>((size_t)Sd * pl.mg.per_sample + 1);
    d.sched = cv.take<int32_t>((size_t)S * nt);
    d.fdt = cv.take<double>((size_t)S * nt);
    d.work = cv.take<unsigned long long>(1);
    d.ir_id = cv.take<int32_t>(N); d.ir_par = cv.take<int32_t>(N);
    d.node_x = cv.take<double>(nn); d.node_y = cv.take<double>(nn); d.seg_L = cv.take<double>(ns);
    d.ir_fixed = cv.take<int8_t>(nn); d.T_ir = cv.take<double>(nn);
    d.up_via = cv.take<int32_t>(nn);
    const int rmax = (c && c->prm.method != EMS_BE) ? 2 * c->prm.krylov_q + 2 : 0;
    if (rmax > 0) {
        d.kr_V = cv.take<unsigned char>((size_t)S * rmax * P * eb);
        d.kr_Ah = cv.take<double>((size_t)S * nt * rmax * rmax);
        d.kr_Ch = cv.take<double>((size_t)S * nt * rmax * rmax);
        d.kr_Lm = cv.take<double>((size_t)S * nt * rmax * rmax);
        d.kr_Xs = cv.take<double>((size_t)S * nt * rmax * (rmax + 1));
        d.kr_sp = cv.take<double>((size_t)S * P); d.kr_sg = cv.take<double>((size_t)S * P);
        d.kr_su = cv.take<double>((size_t)S * P); d.kr_sPf = cv.take<double>((size_t)S * P);
        d.kr_sPb = cv.take<double>((size_t)S * P);
        d.kr_s0 = cv.take<double>((size_t)S * nt);
        d.kr_r = cv.take<int32_t>((size_t)S * nt); d.kr_state = cv.take<int32_t>((size_t)S * nt);
        d.kr_ok = cv.take<int32_t>((size_t)S * nt);
    } else {
        d.kr_V = nullptr;
        d.kr_Ah = d.kr_Ch = d.kr_Lm = d.kr_Xs = nullptr;
        d.kr_sp = d.kr_sg = d.kr_su = d.kr_sPf = d.kr_sPb = d.kr_s0 = nullptr;
        d.kr_r = d.kr_state = d.kr_ok = nullptr;
    }
    return cv.off + 256;
}

template <class T>
cudaError_t up(T *dst, const T *src, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// Chain shapes
// ---------------------------------------------------------------------------
namespace {
int64_t round_warp(int64_t t) { return (t + 31) / 32 * 32; }
bool pow2_chunk(int M) { return M == 4 || M == 8 || M == 16 || M == 32 || M == 64; }
}  // namespace

bool shape_valid(int64_t n, int prec, int kind, int M, int CL, int *T) {
    if (n < 1 || !pow2_chunk(M)) return false;
    const int64_t th = (n + M - 1) / M;             // threads that hold nodes
    int64_t t = round_warp(th);
    switch (kind) {
        case EMS_CHAIN_REGISTER:
            if (prec != EMS_F32 || CL != 1 || t > reg_max_threads(M)) return false;
            break;
        case EMS_CHAIN_SHARED:
            if (prec != EMS_F32 || CL != 1 || t > chain_max_threads(prec, M) ||
                (size_t)5 * sizeof(float) * t * M > kSharedCoefBytes)
                return false;
            break;
        case EMS_CHAIN_GLOBAL:
            if (CL != 1 || t > chain_max_threads(prec, M)) return false;
            break;
        case EMS_CHAIN_CLUSTER: {
            const int tmax = CL >= 2 && CL <= 8 ? cluster_max_threads(prec, M, CL) : 0;
            if (tmax == 0) return false;
            const int64_t tc = round_warp((th + CL - 1) / CL);
            // every CTA must hold nodes of the chain
            if (tc > tmax || th <= (int64_t)(CL - 1) * tc) return false;
            t = tc * CL;
            break;
        }
        case EMS_CHAIN_CLUSTER_SHARED: {
            const int tmax = prec == EMS_F32 && CL >= 2 && CL <= 8 ? cluster_smem_max_threads(M, CL) : 0;
            if (tmax == 0) return false;
            const int64_t tc = round_warp((th + CL - 1) / CL);
            if (tc > tmax || th <= (int64_t)(CL - 1) * tc) return false;
            t = tc * CL;
            break;
        }
        default: return false;
    }
    if (T) *T = (int)t;
    return true;
}

// Built-in choice.  Backward-Euler chains longer than one register-resident
// CTA holds (FP32: 5,120 nodes; FP64: past the streaming kernel's 16,384):
// the smallest cluster that holds them (FP32: 16 nodes per thread, the
// coefficients in shared memory, two CTAs per SM -- 30 % faster than in
// registers on 20,469-node stripes; FP64: 8 per thread).  FP32 chains the
// register kernel holds: 16 nodes per thread (<= 320 threads) for chains of
// more than 2,048 nodes, else 8 (<= 576 threads).  Otherwise the streaming
// kernel with the smallest power-of-two chunk in [4, 64] that keeps the team
// at or below a target (FP32: 448 threads; FP64: 192, the state form keeps
// more per thread), coefficients in shared memory (FP32) while they fit.
// Chains too long for any shape take the branched-tree path.
static void builtin_shape(int64_t n, int prec, int method, int *T, int *M, int *CL, int *kind) {
    *CL = 1;
    const int64_t one_cta = prec == EMS_F32 ? 320 * 16 : 256 * 64;
    const int ck = prec == EMS_F32 ? EMS_CHAIN_CLUSTER_SHARED : EMS_CHAIN_CLUSTER;
    if (method == EMS_BE && n > one_cta)
        for (int cl = 2; cl <= 8; ++cl)
            if (shape_valid(n, prec, ck, cluster_chunk(prec), cl, T)) {
                *M = cluster_chunk(prec); *CL = cl; *kind = ck;
                return;
            }
    if (prec == EMS_F32) {
        const int want = n > 2048 ? 16 : 8;
        for (int m : {want, 16, 8})
            if (shape_valid(n, prec, EMS_CHAIN_REGISTER, m, 1, T)) { *M = m; *kind = EMS_CHAIN_REGISTER; return; }
    }
    const int64_t target = prec == EMS_F32 ? 448 : 192;
    int m = 4;
    while (m < 64 && (n + m - 1) / m > target) m *= 2;
    for (; m <= 64; m *= 2) {
        if (prec == EMS_F32 && shape_valid(n, prec, EMS_CHAIN_SHARED, m, 1, T)) {
            *M = m; *kind = EMS_CHAIN_SHARED;
            return;
        }
        if (shape_valid(n, prec, EMS_CHAIN_GLOBAL, m, 1, T)) { *M = m; *kind = EMS_CHAIN_GLOBAL; return; }
    }
    *T = 0; *M = 0; *kind = 0;
}

void chain_shape(int64_t n, int prec, int method, const std::vector<ems_chain_rule> *rules, int *T, int *M, int *CL,
                 int *kind) {
    if (rules && method == EMS_BE)
        for (const ems_chain_rule &r : *rules)
            if (n >= r.n_lo && n <= r.n_hi && r.kind != EMS_CHAIN_DEFAULT &&
                shape_valid(n, prec, r.kind, r.M, r.CL, T)) {
                *M = r.M; *CL = r.CL; *kind = r.kind;
                return;
            }
    builtin_shape(n, prec, method, T, M, CL, kind);
}

std::vector<ems_chain_rule> shape_candidates(int64_t n, int prec) {
    std::vector<ems_chain_rule> out;
    ems_chain_rule d{n, n, 0, 0, 1, 0};
    builtin_shape(n, prec, EMS_BE, &d.T, &d.M, &d.CL, &d.kind);
    if (d.kind) out.push_back(d);
    auto add = [&](int kind, int M, int CL) {
        ems_chain_rule r{n, n, kind, M, CL, 0};
        if (!shape_valid(n, prec, kind, M, CL, &r.T)) return;
        if (d.kind == kind && d.M == M && d.CL == CL) return;
        out.push_back(r);
    };
    for (int kind : {EMS_CHAIN_REGISTER, EMS_CHAIN_SHARED, EMS_CHAIN_GLOBAL})
        for (int M : {4, 8, 16, 32, 64}) add(kind, M, 1);
    for (int M : {8, 16})
        for (int CL = 2; CL <= 8; ++CL) add(EMS_CHAIN_CLUSTER, M, CL);
    for (int CL = 2; CL <= 8; ++CL) add(EMS_CHAIN_CLUSTER_SHARED, 16, CL);
    return out;
}

}  // namespace ems

using namespace ems;

extern "C" ems_status ems_chain_candidates(int64_t n, int precision, ems_chain_rule *out, int cap, int *count) {
    if (n < 1 || (precision != EMS_F32 && precision != EMS_F64) || cap < 0 || (cap > 0 && !out) || !count)
        return EMS_E_INVAL;
    const std::vector<ems_chain_rule> v = shape_candidates(n, precision);
    const int k = (int)std::min<size_t>(v.size(), (size_t)cap);
    for (int i = 0; i < k; ++i) out[i] = v[i];
    *count = k;
    return EMS_OK;
}

extern "C" ems_status ems_set_chain_rules(ems_ctx *c, const ems_chain_rule *rules, int n_rules) {
    if (!c || n_rules < 0 || (n_rules > 0 && !rules)) return EMS_E_INVAL;
    for (int i = 0; i < n_rules; ++i) {
        const ems_chain_rule &r = rules[i];
        if (r.n_lo < 1 || r.n_hi < r.n_lo) return fail(c, EMS_E_INVAL, "rule range must have 1 <= n_lo <= n_hi");
        if (r.kind < EMS_CHAIN_DEFAULT || r.kind > EMS_CHAIN_CLUSTER_SHARED)
            return fail(c, EMS_E_INVAL, "unknown chain kernel");
        const bool clk = r.kind == EMS_CHAIN_CLUSTER || r.kind == EMS_CHAIN_CLUSTER_SHARED;
        if (r.kind != EMS_CHAIN_DEFAULT && (!pow2_chunk(r.M) || (clk ? (r.CL < 2 || r.CL > 8) : r.CL != 1)))
            return fail(c, EMS_E_INVAL, "M must be 4, 8, 16, 32 or 64; CL 2..8 for a cluster, else 1");
    }
    c->rules.assign(rules, rules + n_rules);
    return EMS_OK;
}

extern "C" size_t ems_workspace_bytes_rules(const ems_params *params, const ems_grid_desc *grid,
                                            const ems_chain_rule *rules, int n_rules) {
    ems_ctx tmp;
    if (!params || n_rules < 0 || (n_rules > 0 && !rules)) return 0;
    tmp.prm = *params;
    if (n_rules > 0 && ems_set_chain_rules(&tmp, rules, n_rules) != EMS_OK) return 0;
    if (!grid) return 0;
    Plan pl;
    if (make_plan(&tmp, params, grid, pl) != EMS_OK) return 0;
    Dev d{};
    const size_t need = carve(&tmp, pl, grid, nullptr, d);
    PlanCache &pc = plan_cache();
    std::lock_guard<std::mutex> lk(pc.mu);
    pc.key = plan_key(params, tmp.rules, grid);
    pc.plan = std::move(pl);
    pc.valid = true;
    return need;
}

extern "C" size_t ems_workspace_bytes(const ems_params *params, const ems_grid_desc *grid) {
    return ems_workspace_bytes_rules(params, grid, nullptr, 0);
}

extern "C" ems_status ems_create(ems_ctx **out, const ems_params *params, void *stream,
                                 void *workspace, size_t ws_bytes) {
    if (!out || !params) return EMS_E_INVAL;
    ems_ctx *c = new ems_ctx();
    c->prm = *params;
    c->stream = (cudaStream_t)stream;
    c->ws = workspace;
    c->ws_bytes = workspace ? ws_bytes : 0;
    c->own_ws = workspace == nullptr;
    if (workspace && ((uintptr_t)workspace & 255)) {
        delete c;
        return EMS_E_INVAL;
    }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        cluster_smem_init() != cudaSuccess) {
        if (c->ev0) cudaEventDestroy(c->ev0);
        if (c->ev1) cudaEventDestroy(c->ev1);
        delete c;
        return EMS_E_CUDA;
    }
    *out = c;
    return EMS_OK;
}

extern "C" ems_status ems_destroy(ems_ctx *c) {
    if (!c) return EMS_E_INVAL;
    for (auto &b : c->buckets)
        if (b.d_trees) cudaFree(b.d_trees);
    if (c->ttf_graph) cudaGraphExecDestroy(c->ttf_graph);
    for (auto e : c->gev) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
    return EMS_OK;
}

extern "C" const char *ems_last_error(const ems_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" ems_status ems_load_grid(ems_ctx *c, const ems_grid_desc *g) {
    if (!c) return EMS_E_INVAL;
    if (!g) return fail(c, EMS_E_INVAL, "null grid");
    Plan pl;
    bool cached = false;
    {
        PlanCache &pc = plan_cache();
        std::lock_guard<std::mutex> lk(pc.mu);
        if (pc.valid) {
            if (pc.key == plan_key(&c->prm, c->rules, g)) {
                pl = std::move(pc.plan);
                cached = true;
            }
            pc.plan = Plan();
            pc.valid = false;
        }
    }
    if (cached) EMS_TRY(validate(c, &c->prm, g));     // the factors and the map are not in the key
    else EMS_TRY(make_plan(c, &c->prm, g, pl));
    Dev d{};
    size_t need = carve(c, pl, g, nullptr, d);
    if (c->own_ws) {
        if (c->ws && c->ws_bytes < need) { cudaFree(c->ws); c->ws = nullptr; }
        if (!c->ws) {
            if (cudaMalloc(&c->ws, need) != cudaSuccess)
                return fail(c, EMS_E_NOMEM, "workspace allocation failed");
            c->ws_bytes = need;
        }
    } else if (c->ws_bytes < need) {
        return fail(c, EMS_E_NOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
    }
    carve(c, pl, g, c->ws, c->d);
    Dev &D = c->d;
    cudaStream_t st = c->stream;
    EMS_CUDA(c, cudaMemsetAsync(c->ws, 0, need - 256, st));
    {   // polls a grid-barrier wait makes before giving up (words 2-3 of the barrier block)
        const long long lim = kDefaultWaitLimit;
        EMS_CUDA(c, cudaMemcpyAsync(D.gbar + 2, &lim, sizeof lim, cudaMemcpyHostToDevice, st));
        EMS_CUDA(c, cudaStreamSynchronize(st));
    }
    c->S = pl.S; c->S_all = pl.S; c->W = pl.Sd; c->win_s0 = 0;
    c->d_all = c->d;
    c->n_nodes = g->n_nodes; c->n_seg = g->n_seg; c->n_pads = g->n_pads;
    c->n_sinks = g->n_sinks; c->nf = (int)pl.ir.node_of_free.size(); c->nnz = (int64_t)pl.ir.col.size();
    c->N = pl.tr.off.back(); c->P = pl.P; c->n_trees = pl.tr.n_trees;
    c->maxv = c->prm.max_voids_per_tree;
    c->rmax = c->prm.method != EMS_BE ? 2 * c->prm.krylov_q + 2 : 0;
    const int S = c->S, ns = c->n_seg;
    // grid
    EMS_CUDA(c, up(D.seg_a, g->seg_a, ns, st)); EMS_CUDA(c, up(D.seg_b, g->seg_b, ns, st));
    EMS_CUDA(c, up(D.seg_R0, g->seg_R0, ns, st)); EMS_CUDA(c, up(D.seg_W, g->seg_W, ns, st));
    EMS_CUDA(c, up(D.seg_H, g->seg_H, ns, st));
    // per-sample copies of one host row: upload sample 0, replicate on the device
    auto replicate = [&](double *dst, const double *row, size_t n) -> ems_status {
        EMS_CUDA(c, up(dst, row, n, st));
        for (int s = 1; s < S; ++s)
            EMS_CUDA(c, cudaMemcpyAsync(dst + (size_t)s * n, dst, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        return EMS_OK;
    };
    EMS_TRY(replicate(D.R, g->seg_R0, ns));
    EMS_TRY(replicate(D.R_prev, g->seg_R0, ns));
    {
        std::vector<double> ones((g->kappa_factor && g->sigc_factor) ? 0 : (size_t)ns, 1.0);
        if (g->kappa_factor) EMS_CUDA(c, up(D.kfac, g->kappa_factor, (size_t)S * ns, st));
        else EMS_TRY(replicate(D.kfac, ones.data(), ns));
        if (g->sigc_factor) EMS_CUDA(c, up(D.sfac, g->sigc_factor, (size_t)S * ns, st));
        else EMS_TRY(replicate(D.sfac, ones.data(), ns));
        EMS_CUDA(c, cudaStreamSynchronize(st));
    }
    // IR
    const HostIR &ir = pl.ir;
    EMS_CUDA(c, up(D.ir_free_of_node, ir.free_of_node.data(), ir.free_of_node.size(), st));
    EMS_CUDA(c, up(D.ir_node_of_free, ir.node_of_free.data(), ir.node_of_free.size(), st));
    EMS_CUDA(c, up(D.csr_ptr, ir.ptr.data(), ir.ptr.size(), st));
    EMS_CUDA(c, up(D.csr_col, ir.col.data(), ir.col.size(), st));
    EMS_CUDA(c, up(D.ent_ptr, ir.ent_ptr.data(), ir.ent_ptr.size(), st));
    EMS_CUDA(c, up(D.ent_seg, ir.ent_seg.data(), ir.ent_seg.size(), st));
    EMS_CUDA(c, up(D.ent_diag, ir.ent_diag.data(), ir.ent_diag.size(), st));
    EMS_CUDA(c, up(D.rhs_ptr, ir.rhs_ptr.data(), ir.rhs_ptr.size(), st));
    EMS_CUDA(c, up(D.rhs_seg, ir.rhs_seg.data(), ir.rhs_seg.size(), st));
    EMS_CUDA(c, up(D.rhs_padV, ir.rhs_padV.data(), ir.rhs_padV.size(), st));
    EMS_CUDA(c, up(D.sink_of_free, ir.sink.data(), ir.sink.size(), st));
    EMS_CUDA(c, up(D.pad_V_of_node, ir.padV_of_node.data(), ir.padV_of_node.size(), st));
    // multigrid hierarchy of the IR system (built from R0 in make_plan)
    c->mg = MGDevice();
    c->mg_blocks = 0;
    if (pl.mg.L >= 2) {
        EMS_CUDA(c, up(D.mg_i, pl.mg.ints.data(), pl.mg.ints.size(), st));
        EMS_CUDA(c, up(D.mg_d, pl.mg.dbls.data(), pl.mg.dbls.size(), st));
        {
            const std::vector<float> f(pl.mg.dbls.begin(), pl.mg.dbls.end());
            EMS_CUDA(c, up(D.mg_f, f.data(), f.size(), st));
            EMS_CUDA(c, cudaStreamSynchronize(st));    // f is a host temporary
        }
        c->mg.L = pl.mg.L;
        for (int l = 0; l < EMS_MG_MAXLV; ++l) c->mg.lv[l] = pl.mg.lv[l];
        c->mg.cinv = pl.mg.cinv;
        c->mg.per_sample = pl.mg.per_sample;
        c->mg.I = D.mg_i;
        c->mg.D = D.mg_d;
        c->mg.F = D.mg_f;
        c->mg.scratch = D.mg_sc;
    }
    // initial guess: every free node at the mean pad voltage
    {
        double vm = 0.0;
        for (int i = 0; i < g->n_pads; ++i) vm += g->pad_V[i];
        vm /= g->n_pads;
        std::vector<double> x0((size_t)c->nf, vm), u0((size_t)g->n_nodes);
        for (int i = 0; i < g->n_nodes; ++i) u0[i] = std::isnan(ir.padV_of_node[i]) ? vm : ir.padV_of_node[i];
        // with windows the IR guess is gathered from u before every solve
        if (!windowed(c)) EMS_TRY(replicate(D.ir_x, x0.data(), x0.size()));
        EMS_TRY(replicate(D.u, u0.data(), u0.size()));
        EMS_CUDA(c, cudaStreamSynchronize(st));
    }
    // trees
    HostTrees &tr = pl.tr;
    const int64_t N = c->N;
    EMS_CUDA(c, up(D.toff, tr.off.data(), tr.off.size(), st));
    {   // parents and children as global node indices
        std::vector<int32_t> gp(N), gc(tr.child_idx.size());
        for (int t = 0; t < tr.n_trees; ++t)
            for (int64_t i = tr.off[t]; i < tr.off[t + 1]; ++i) {
                gp[i] = tr.par[i] < 0 ? -1 : (int32_t)(tr.off[t] + tr.par[i]);
                for (int k = tr.child_ptr[i]; k < tr.child_ptr[i + 1]; ++k)
                    gc[k] = (int32_t)(tr.off[t] + tr.child_idx[k]);
            }
        EMS_CUDA(c, up(D.par, gp.data(), N, st));
        EMS_CUDA(c, up(D.child_idx, gc.data(), gc.size(), st));
        EMS_CUDA(c, cudaStreamSynchronize(st));   // gp / gc are host temporaries
    }
    EMS_CUDA(c, up(D.face_seg, tr.face_seg.data(), N, st));
    EMS_CUDA(c, up(D.owner_seg, tr.owner_seg.data(), N, st));
    EMS_CUDA(c, up(D.inc_seg, tr.inc_seg.data(), tr.inc_seg.size(), st));
    EMS_CUDA(c, up(D.child_ptr, tr.child_ptr.data(), tr.child_ptr.size(), st));
    EMS_CUDA(c, up(D.face_sign, tr.face_sign.data(), N, st));
    EMS_CUDA(c, up(D.face_dx, tr.face_dx.data(), N, st));
    EMS_CUDA(c, up(D.face_area, tr.face_area.data(), N, st));
    EMS_CUDA(c, up(D.nx_, tr.x.data(), N, st));
    EMS_CUDA(c, up(D.ny_, tr.y.data(), N, st));
    EMS_CUDA(c, up(D.ir_id, tr.ir_id.data(), N, st));
    EMS_CUDA(c, up(D.ir_par, tr.ir_par.data(), N, st));
    EMS_CUDA(c, up(D.node_x, g->node_x, (size_t)g->n_nodes, st));
    EMS_CUDA(c, up(D.node_y, g->node_y, (size_t)g->n_nodes, st));
    EMS_CUDA(c, up(D.seg_L, g->seg_L, (size_t)ns, st));
    {   // IR nodes whose temperature is given: vias between layers and pads
        std::vector<int32_t> lay0((size_t)g->n_nodes, -1);
        std::vector<int8_t> fixed((size_t)g->n_nodes, 0);
        for (int q = 0; q < ns; ++q)
            for (int32_t nd : {g->seg_a[q], g->seg_b[q]}) {
                if (lay0[nd] < 0) lay0[nd] = g->seg_layer[q];
                else if (lay0[nd] != g->seg_layer[q]) fixed[nd] = 1;
            }
        for (int q = 0; q < g->n_pads; ++q) fixed[g->pad_node[q]] = 1;
        EMS_CUDA(c, up(D.ir_fixed, fixed.data(), fixed.size(), st));
        // the via from each IR node up to a strictly higher layer (-1: none);
        // a node's layer is the layer of its wire segments
        std::vector<int32_t> nl((size_t)g->n_nodes, -1), upv((size_t)g->n_nodes, -1);
        if (g->seg_via) {
            for (int q = 0; q < ns; ++q)
                if (!g->seg_via[q]) { nl[g->seg_a[q]] = g->seg_layer[q]; nl[g->seg_b[q]] = g->seg_layer[q]; }
            for (int q = 0; q < ns; ++q) {
                if (!g->seg_via[q]) continue;
                const int32_t ea = g->seg_a[q], eb = g->seg_b[q];
                if (nl[ea] >= 0 && nl[eb] > nl[ea] && upv[ea] < 0) upv[ea] = q;
                if (nl[eb] >= 0 && nl[ea] > nl[eb] && upv[eb] < 0) upv[eb] = q;
            }
        }
        EMS_CUDA(c, up(D.up_via, upv.data(), upv.size(), st));
        EMS_CUDA(c, cudaStreamSynchronize(st));
    }
    {   // inc_ptr is per node: global CSR over all nodes
        EMS_CUDA(c, up(D.inc_ptr, tr.inc_ptr.data(), tr.inc_ptr.size(), st));
    }
    std::vector<int64_t> pb(c->n_trees);
    std::vector<int32_t> pT(c->n_trees), pM(c->n_trees);
    for (int t = 0; t < c->n_trees; ++t) { pb[t] = pl.pack[t].pbase; pT[t] = pl.pack[t].T; pM[t] = pl.pack[t].M; }
    EMS_CUDA(c, up(D.pbase, pb.data(), pb.size(), st));
    EMS_CUDA(c, up(D.pT, pT.data(), pT.size(), st));
    EMS_CUDA(c, up(D.pM, pM.data(), pM.size(), st));
    // buckets by (chain, T, M)
    for (auto &b : c->buckets)
        if (b.d_trees) cudaFree(b.d_trees);
    c->buckets.clear();
    for (int t = 0; t < c->n_trees; ++t) {
        bool ch = pl.pack[t].T > 1;
        Bucket *bk = nullptr;
        for (auto &b : c->buckets)
            if (b.chain == ch && (!ch || (b.T == pl.pack[t].T && b.M == pl.pack[t].M && b.CL == pl.pack[t].CL &&
                                          b.kind == pl.pack[t].kind)))
                bk = &b;
        if (!bk) {
            c->buckets.push_back(Bucket{});
            bk = &c->buckets.back();
            bk->chain = ch; bk->T = ch ? pl.pack[t].T : 1; bk->M = ch ? pl.pack[t].M : 0;
            bk->CL = ch ? pl.pack[t].CL : 1;
            bk->kind = ch ? pl.pack[t].kind : 0;
        }
        bk->trees.push_back(t);
    }
    for (auto &b : c->buckets) {
        EMS_CUDA(c, cudaMalloc(&b.d_trees, b.trees.size() * sizeof(int32_t)));
        EMS_CUDA(c, up(b.d_trees, b.trees.data(), b.trees.size(), st));
    }
    c->trees = std::move(pl.tr);
    c->pack = std::move(pl.pack);
    if (c->ttf_graph) { cudaGraphExecDestroy(c->ttf_graph); c->ttf_graph = nullptr; }
    c->t = 0.0;
    c->factored_dt = -1.0;
    c->have_u = false;
    c->joule = false;
    c->pnx = c->pny = 0;
    c->loaded = true;
    // uniform temperature, node physics, initial stress
    EMS_TRY(ems_set_thermal_map(c, nullptr, 0, 0, 0, 0, 0, 0));
    EMS_TRY(ems::init_sigma(c));
    EMS_CUDA(c, cudaStreamSynchronize(st));
    return EMS_OK;
}

extern "C" ems_status ems_set_wait_limit(ems_ctx *c, long long polls) {
    if (!c || polls < 0) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    const long long lim = polls == 0 ? kDefaultWaitLimit : polls;
    EMS_CUDA(c, cudaMemcpyAsync(c->d_all.gbar + 2, &lim, sizeof lim, cudaMemcpyHostToDevice, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_dims(const ems_ctx *c, int *n_trees, int64_t *n_stress_nodes, int *n_samples) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return EMS_E_STATE;
    if (n_trees) *n_trees = c->n_trees;
    if (n_stress_nodes) *n_stress_nodes = c->N;
    if (n_samples) *n_samples = c->S;
    return EMS_OK;
}

extern "C" ems_status ems_launch_count(const ems_ctx *c, int64_t *launches) {
    if (!c || !launches) return EMS_E_INVAL;
    *launches = c->launches;
    return EMS_OK;
}

extern "C" ems_status ems_get_currents(ems_ctx *c, double *j) {
    if (!c || !j) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    EMS_CUDA(c, cudaMemcpyAsync(j, c->d.j, sizeof(double) * c->S * c->n_seg, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_get_resistance(ems_ctx *c, double *R) {
    if (!c || !R) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    EMS_CUDA(c, cudaMemcpyAsync(R, c->d.R, sizeof(double) * c->S * c->n_seg, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_get_sigma(ems_ctx *c, double *sigma) {
    if (!c || !sigma) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    return ems::each_window(c, [&](int s0, int ns) -> ems_status {
        EMS_TRY(ems::pack_sigma(c, /*to_packed=*/false));   // packed -> canonical (scratch)
        EMS_CUDA(c, cudaMemcpyAsync(sigma + (size_t)s0 * c->N, c->d.sig_ss, sizeof(double) * ns * c->N,
                                    cudaMemcpyDeviceToHost, c->stream));
        EMS_CUDA(c, cudaStreamSynchronize(c->stream));
        return EMS_OK;
    });
}

extern "C" ems_status ems_get_voids(ems_ctx *c, int cap, int32_t *sample, int32_t *node, int32_t *seg,
                                    double *volume, double *t_nuc, int *n) {
    if (!c || !n) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    const size_t st_n = (size_t)c->S * c->n_trees, mv = c->maxv;
    std::vector<int32_t> cnt(st_n), vn(st_n * mv), vs(st_n * mv);
    std::vector<double> vv(st_n * mv), vt(st_n * mv);
    auto cs = c->stream;
    EMS_CUDA(c, cudaMemcpyAsync(cnt.data(), c->d.v_count, st_n * 4, cudaMemcpyDeviceToHost, cs));
    EMS_CUDA(c, cudaMemcpyAsync(vn.data(), c->d.v_node, st_n * mv * 4, cudaMemcpyDeviceToHost, cs));
    EMS_CUDA(c, cudaMemcpyAsync(vs.data(), c->d.v_seg, st_n * mv * 4, cudaMemcpyDeviceToHost, cs));
    EMS_CUDA(c, cudaMemcpyAsync(vv.data(), c->d.v_vol, st_n * mv * 8, cudaMemcpyDeviceToHost, cs));
    EMS_CUDA(c, cudaMemcpyAsync(vt.data(), c->d.v_tnuc, st_n * mv * 8, cudaMemcpyDeviceToHost, cs));
    EMS_CUDA(c, cudaStreamSynchronize(cs));
    int k = 0;
    for (int s = 0; s < c->S; ++s)
        for (int t = 0; t < c->n_trees; ++t) {
            size_t st = (size_t)s * c->n_trees + t;
            for (int q = 0; q < cnt[st]; ++q) {
                if (k < cap) {
                    size_t e = st * mv + q;
                    if (sample) sample[k] = s;
                    if (node) node[k] = (int32_t)(c->trees.off[t] + vn[e]);
                    if (seg) seg[k] = vs[e];
                    if (volume) volume[k] = vv[e];
                    if (t_nuc) t_nuc[k] = vt[e];
                }
                ++k;
            }
        }
    *n = k;
    return EMS_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint: header + sigma (canonical, double) + void tables + R + u + x
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    uint64_t magic, S, N, n_trees, maxv, n_seg, n_nodes, nf;
    double t;
};
const uint64_t kMagic = 0x454d5333434b5054ull;  // "EMS3CKPT"
}  // namespace

extern "C" ems_status ems_state_export(ems_ctx *c, void *buf, size_t *bytes) {
    if (!c || !bytes) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    const size_t S = c->S, N = c->N, st = S * c->n_trees, mv = c->maxv;
    const size_t need = sizeof(CkptHeader) + S * N * 8 + st * 4 + st * mv * (4 + 4 + 8 + 8) +
                        S * c->n_seg * 8 + S * c->n_nodes * 8 + S * c->nf * 8;
    if (!buf) { *bytes = need; return EMS_OK; }
    if (*bytes < need) return fail(c, EMS_E_INVAL, "checkpoint buffer too small");
    char *p = (char *)buf;
    CkptHeader h{kMagic, S, N, (uint64_t)c->n_trees, mv, (uint64_t)c->n_seg, (uint64_t)c->n_nodes,
                 (uint64_t)c->nf, c->t};
    std::memcpy(p, &h, sizeof h); p += sizeof h;
    EMS_TRY(ems_get_sigma(c, (double *)p)); p += S * N * 8;
    auto cs = c->stream;
    auto dn = [&](void *dst, const void *src, size_t nb) {
        return cudaMemcpyAsync(dst, src, nb, cudaMemcpyDeviceToHost, cs);
    };
    EMS_CUDA(c, dn(p, c->d.v_count, st * 4)); p += st * 4;
    EMS_CUDA(c, dn(p, c->d.v_node, st * mv * 4)); p += st * mv * 4;
    EMS_CUDA(c, dn(p, c->d.v_seg, st * mv * 4)); p += st * mv * 4;
    EMS_CUDA(c, dn(p, c->d.v_vol, st * mv * 8)); p += st * mv * 8;
    EMS_CUDA(c, dn(p, c->d.v_tnuc, st * mv * 8)); p += st * mv * 8;
    EMS_CUDA(c, dn(p, c->d.R, S * c->n_seg * 8)); p += S * c->n_seg * 8;
    EMS_CUDA(c, dn(p, c->d.u, S * c->n_nodes * 8)); p += S * c->n_nodes * 8;
    if (!windowed(c)) {
        EMS_CUDA(c, dn(p, c->d.ir_x, S * c->nf * 8));
    } else {
        // windows: the IR guess is the free nodes' voltages
        char *px = p;
        EMS_TRY(each_window(c, [&](int s0, int ns) -> ems_status {
            EMS_TRY(gather_x(c));
            EMS_CUDA(c, dn(px + (size_t)s0 * c->nf * 8, c->d.ir_x, (size_t)ns * c->nf * 8));
            EMS_CUDA(c, cudaStreamSynchronize(cs));
            return EMS_OK;
        }));
    }
    p += S * c->nf * 8;
    EMS_CUDA(c, cudaStreamSynchronize(cs));
    *bytes = need;
    return EMS_OK;
}

extern "C" ems_status ems_state_import(ems_ctx *c, const void *buf, size_t bytes) {
    if (!c || !buf) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    CkptHeader h;
    if (bytes < sizeof h) return fail(c, EMS_E_INVAL, "checkpoint truncated");
    std::memcpy(&h, buf, sizeof h);
    const size_t S = c->S, N = c->N, st = S * c->n_trees, mv = c->maxv;
    if (h.magic != kMagic || h.S != S || h.N != N || h.n_trees != (uint64_t)c->n_trees || h.maxv != mv ||
        h.n_seg != (uint64_t)c->n_seg || h.n_nodes != (uint64_t)c->n_nodes || h.nf != (uint64_t)c->nf)
        return fail(c, EMS_E_INVAL, "checkpoint does not match the loaded grid");
    const size_t need = sizeof(CkptHeader) + S * N * 8 + st * 4 + st * mv * (4 + 4 + 8 + 8) +
                        S * c->n_seg * 8 + S * c->n_nodes * 8 + S * c->nf * 8;
    if (bytes < need) return fail(c, EMS_E_INVAL, "checkpoint truncated");
    const char *p = (const char *)buf + sizeof h;
    auto cs = c->stream;
    auto upb = [&](void *dst, const void *src, size_t nb) {
        return cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, cs);
    };
    const char *psig = p;
    p += S * N * 8;
    EMS_CUDA(c, upb(c->d.v_count, p, st * 4)); p += st * 4;
    EMS_CUDA(c, upb(c->d.v_node, p, st * mv * 4)); p += st * mv * 4;
    EMS_CUDA(c, upb(c->d.v_seg, p, st * mv * 4)); p += st * mv * 4;
    EMS_CUDA(c, upb(c->d.v_vol, p, st * mv * 8)); p += st * mv * 8;
    EMS_CUDA(c, upb(c->d.v_tnuc, p, st * mv * 8)); p += st * mv * 8;
    EMS_CUDA(c, upb(c->d.R, p, S * c->n_seg * 8)); p += S * c->n_seg * 8;
    EMS_CUDA(c, upb(c->d.u, p, S * c->n_nodes * 8)); p += S * c->n_nodes * 8;
    if (!windowed(c)) EMS_CUDA(c, upb(c->d.ir_x, p, S * c->nf * 8));   // windows: gathered from u
    p += S * c->nf * 8;
    c->t = h.t;
    c->have_u = true;
    EMS_CUDA(c, cudaStreamSynchronize(cs));
    // stress through the canonical scratch, one window at a time; thresholds
    // with the imported voids (every tree marked for a refactor)
    return each_window(c, [&](int s0, int ns) -> ems_status {
        EMS_CUDA(c, upb(c->d.sig_ss, psig + (size_t)s0 * N * 8, (size_t)ns * N * 8));
        EMS_TRY(ems::node_physics(c));
        EMS_TRY(ems::pack_sigma(c, /*to_packed=*/true));
        EMS_TRY(ems::ir_currents_and_drop(c));
        EMS_CUDA(c, cudaStreamSynchronize(cs));
        return EMS_OK;
    });
}
