// ems_spice.cu -- SPICE power-grid netlist reader (host code).
//
// The paper's flow converts each design's power-grid netlist (PNA output) to
// SPICE, keeps every via resistor, and extracts the interconnect trees from
// the resistors (Sec. IV-A, IV-C).  This reader turns such a netlist into an
// ems_grid_desc: resistors between two nodes of one metal layer are wire
// segments, resistors between nodes of different layers are vias,
// node-to-ground voltage sources are pads and node-to-ground current sources
// are sinks.  Node names carry their layer and position, n<layer>_<x>_<y>
// with integer coordinates in units of opts->coord_unit (metres), the naming
// of the common power-grid benchmark netlists.
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "ems_internal.cuh"

struct ems_netlist {
    std::vector<double> node_x, node_y;
    std::vector<int32_t> node_layer;
    std::vector<int32_t> seg_a, seg_b, seg_layer, seg_cells;
    std::vector<double> seg_R0, seg_W, seg_H, seg_L;
    std::vector<int8_t> seg_via;
    std::vector<int32_t> pad_node, sink_node;
    std::vector<double> pad_V, sink_I;
    std::string err;
};

namespace {

bool parse_node(const std::string &name, int *layer, long long *x, long long *y) {
    // n<layer>_<x>_<y>
    if (name.size() < 6 || (name[0] != 'n' && name[0] != 'N')) return false;
    const char *p = name.c_str() + 1;
    char *end = nullptr;
    const long l = strtol(p, &end, 10);
    if (end == p || *end != '_' || l < 1 || l > 64) return false;
    p = end + 1;
    const long long xx = strtoll(p, &end, 10);
    if (end == p || *end != '_') return false;
    p = end + 1;
    const long long yy = strtoll(p, &end, 10);
    if (end == p || *end != '\0') return false;
    *layer = (int)l;
    *x = xx;
    *y = yy;
    return true;
}

bool is_ground(const std::string &s) {
    return s == "0" || s == "gnd" || s == "GND";
}

bool parse_value(const std::string &s, double *v) {
    char *end = nullptr;
    const double d = strtod(s.c_str(), &end);
    if (end == s.c_str() || !std::isfinite(d)) return false;
    *v = d;
    return *end == '\0';
}

}  // namespace

extern "C" ems_status ems_spice_parse(const char *text, size_t len, const ems_spice_opts *o, ems_netlist **out) {
    if (!text || !o || !out || !o->W || !o->H || o->n_layers < 1 || o->n_layers > 64 || !(o->coord_unit > 0.0) ||
        !(o->dx > 0.0) || !(o->via_W > 0.0) || !(o->via_H > 0.0))
        return EMS_E_INVAL;
    for (int l = 0; l < o->n_layers; ++l)
        if (!(o->W[l] > 0.0) || !(o->H[l] > 0.0)) return EMS_E_INVAL;
    *out = nullptr;
    ems_netlist *nl = new ems_netlist();
    std::unordered_map<std::string, int32_t> id;
    auto node = [&](const std::string &name, int32_t *idx) -> bool {
        auto it = id.find(name);
        if (it != id.end()) { *idx = it->second; return true; }
        int layer;
        long long x, y;
        if (!parse_node(name, &layer, &x, &y) || layer > o->n_layers) return false;
        *idx = (int32_t)nl->node_x.size();
        id.emplace(name, *idx);
        nl->node_x.push_back((double)x * o->coord_unit);
        nl->node_y.push_back((double)y * o->coord_unit);
        nl->node_layer.push_back(layer);
        return true;
    };
    size_t pos = 0;
    int line_no = 0;
    auto bad = [&](const std::string &why) {
        nl->err = "line " + std::to_string(line_no) + ": " + why;
        return EMS_E_INVAL;
    };
    ems_status st = EMS_OK;
    while (pos < len && st == EMS_OK) {
        size_t e = pos;
        while (e < len && text[e] != '\n') ++e;
        std::string line(text + pos, e - pos);
        pos = e + 1;
        ++line_no;
        // tokens
        std::vector<std::string> tok;
        for (size_t k = 0; k < line.size();) {
            while (k < line.size() && std::isspace((unsigned char)line[k])) ++k;
            size_t b = k;
            while (k < line.size() && !std::isspace((unsigned char)line[k])) ++k;
            if (k > b) tok.emplace_back(line.substr(b, k - b));
        }
        if (tok.empty() || tok[0][0] == '*' || tok[0][0] == '.') continue;
        const char kind = (char)std::toupper((unsigned char)tok[0][0]);
        if (tok.size() != 4) { st = bad("expected: name node node value"); break; }
        double val;
        if (!parse_value(tok[3], &val)) { st = bad("bad value '" + tok[3] + "'"); break; }
        const bool g1 = is_ground(tok[1]), g2 = is_ground(tok[2]);
        if (kind == 'R') {
            int32_t a, b;
            if (g1 || g2) { st = bad("resistor to ground"); break; }
            if (!node(tok[1], &a) || !node(tok[2], &b)) { st = bad("node name is not n<layer>_<x>_<y>"); break; }
            if (a == b || !(val > 0.0)) { st = bad("resistor needs two nodes and R > 0"); break; }
            const int la = nl->node_layer[a], lb = nl->node_layer[b];
            nl->seg_a.push_back(a);
            nl->seg_b.push_back(b);
            nl->seg_R0.push_back(val);
            if (la == lb) {
                const double L = std::hypot(nl->node_x[b] - nl->node_x[a], nl->node_y[b] - nl->node_y[a]);
                if (!(L > 0.0)) { st = bad("wire of zero length"); break; }
                nl->seg_layer.push_back(la);
                nl->seg_W.push_back(o->W[la - 1]);
                nl->seg_H.push_back(o->H[la - 1]);
                nl->seg_L.push_back(L);
                nl->seg_cells.push_back((int32_t)std::max(1.0, std::floor(L / o->dx + 0.5)));
                nl->seg_via.push_back(0);
            } else {
                nl->seg_layer.push_back(std::min(la, lb));
                nl->seg_W.push_back(o->via_W);
                nl->seg_H.push_back(o->via_H);
                nl->seg_L.push_back(o->via_H);
                nl->seg_cells.push_back(1);
                nl->seg_via.push_back(1);
            }
        } else if (kind == 'V' || kind == 'I') {
            if (g1 == g2) { st = bad("source must join a node and ground"); break; }
            int32_t a;
            if (!node(g1 ? tok[2] : tok[1], &a)) { st = bad("node name is not n<layer>_<x>_<y>"); break; }
            // V n 0 v: node at +v; I n 0 i: i flows out of n into ground (a sink)
            const double sgn = g1 ? -1.0 : 1.0;
            if (kind == 'V') { nl->pad_node.push_back(a); nl->pad_V.push_back(sgn * val); }
            else { nl->sink_node.push_back(a); nl->sink_I.push_back(sgn * val); }
        } else {
            st = bad(std::string("unsupported element '") + tok[0] + "'");
        }
    }
    if (st == EMS_OK && (nl->seg_a.empty() || nl->pad_node.empty())) {
        nl->err = "netlist needs resistors and at least one voltage source";
        st = EMS_E_INVAL;
    }
    *out = nl;        // also on error: ems_netlist_error() tells why
    return st;
}

extern "C" ems_status ems_netlist_desc(const ems_netlist *nl, ems_grid_desc *d) {
    if (!nl || !d) return EMS_E_INVAL;
    std::memset(d, 0, sizeof *d);
    d->n_nodes = (int)nl->node_x.size();
    d->node_x = nl->node_x.data();
    d->node_y = nl->node_y.data();
    d->n_seg = (int)nl->seg_a.size();
    d->seg_a = nl->seg_a.data();
    d->seg_b = nl->seg_b.data();
    d->seg_layer = nl->seg_layer.data();
    d->seg_cells = nl->seg_cells.data();
    d->seg_R0 = nl->seg_R0.data();
    d->seg_W = nl->seg_W.data();
    d->seg_H = nl->seg_H.data();
    d->seg_L = nl->seg_L.data();
    d->n_pads = (int)nl->pad_node.size();
    d->pad_node = nl->pad_node.data();
    d->pad_V = nl->pad_V.data();
    d->n_sinks = (int)nl->sink_node.size();
    d->sink_node = nl->sink_node.data();
    d->sink_I = nl->sink_I.data();
    d->n_samples = 0;
    d->seg_via = nl->seg_via.data();
    return EMS_OK;
}

extern "C" const char *ems_netlist_error(const ems_netlist *nl) { return nl ? nl->err.c_str() : "null netlist"; }

extern "C" void ems_netlist_free(ems_netlist *nl) { delete nl; }
