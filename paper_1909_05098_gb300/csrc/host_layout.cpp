// Host side of the pre-computation: internal element/node order and the
// node -> element-slot gather structure (cold path, integer work only).
//
// The paper's time loop is two parallel-for loops, over elements and then
// over nodes (Algorithm 1, Section 2.4), with the element loads "added to the
// global nodal loads" (Eq. 11).  Here that addition is a gather: every free
// node owns the list of (element, corner) slots it receives a load from,
// sorted by INPUT element id, so the floating-point sum order is fixed by the
// caller's mesh alone and is the same for every internal order and launch
// shape.  No float atomics are used anywhere.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <queue>
#include <string>

#include "fedfem_internal.h"

namespace fedfem {
namespace {

uint64_t spread3(uint64_t v) {   // 21 bits -> every third of 63 bits
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

// Keep element groups (independent meshes) apart: stable sort by group.
void group_sort(const MeshInput& in, std::vector<int32_t>& elem_of) {
    if (!in.groups) return;
    const std::vector<int32_t>& g = *in.groups;
    std::stable_sort(elem_of.begin(), elem_of.end(), [&](int32_t a, int32_t b) { return g[a] < g[b]; });
}

void morton_order(const MeshInput& in, std::vector<int32_t>& elem_of) {
    const int nv = in.nv;
    std::vector<double> c(3 * in.E);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t e = 0; e < in.E; ++e) {
        for (int d = 0; d < 3; ++d) {
            double s = 0;
            for (int k = 0; k < nv; ++k) s += in.xyz[3 * (int64_t)in.conn[e * nv + k] + d];
            s /= nv;
            c[3 * e + d] = s;
            lo[d] = std::min(lo[d], s);
            hi[d] = std::max(hi[d], s);
        }
    }
    double span = 0;
    for (int d = 0; d < 3; ++d) span = std::max(span, hi[d] - lo[d]);
    const double scale = span > 0 ? 2097151.0 / span : 0.0;   // one scale keeps cells cubic
    std::vector<std::pair<uint64_t, int32_t>> key(in.E);
    for (int64_t e = 0; e < in.E; ++e) {
        uint64_t q[3];
        for (int d = 0; d < 3; ++d) {
            double v = (c[3 * e + d] - lo[d]) * scale;
            q[d] = (uint64_t)std::min(2097151.0, std::max(0.0, v));
        }
        key[e] = {spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2), (int32_t)e};
    }
    std::sort(key.begin(), key.end());
    for (int64_t e = 0; e < in.E; ++e) elem_of[e] = key[e].second;
}

// Reverse Cuthill-McKee on the node graph (nodes sharing an element), started
// from a pseudo-peripheral node found by repeated breadth-first search
// (George & Liu).  Elements are then ordered by their smallest node label.
void rcm_order(const MeshInput& in, std::vector<int32_t>& elem_of) {
    const int nv = in.nv;
    const int64_t N = in.N, E = in.E;
    std::vector<int64_t> off(N + 1, 0);
    for (int64_t i = 0; i < E * nv; ++i) off[in.conn[i] + 1]++;
    for (int64_t i = 0; i < N; ++i) off[i + 1] += off[i];
    std::vector<int32_t> inc(E * nv);
    {
        std::vector<int64_t> pos(off.begin(), off.end() - 1);
        for (int64_t e = 0; e < E; ++e)
            for (int k = 0; k < nv; ++k) inc[pos[in.conn[e * nv + k]]++] = (int32_t)e;
    }
    std::vector<int64_t> aoff(N + 1, 0);
    std::vector<int32_t> adj;
    {
        std::vector<int32_t> tmp;
        for (int64_t n = 0; n < N; ++n) {
            tmp.clear();
            for (int64_t p = off[n]; p < off[n + 1]; ++p)
                for (int k = 0; k < nv; ++k) {
                    int32_t m = in.conn[(int64_t)inc[p] * nv + k];
                    if (m != n) tmp.push_back(m);
                }
            std::sort(tmp.begin(), tmp.end());
            tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
            adj.insert(adj.end(), tmp.begin(), tmp.end());
            aoff[n + 1] = (int64_t)adj.size();
        }
    }
    auto deg = [&](int64_t n) { return aoff[n + 1] - aoff[n]; };
    std::vector<int32_t> label(N, -1);
    int32_t next = 0;
    std::vector<int32_t> level(N, -1);
    for (int64_t seed = 0; seed < N; ++seed) {
        if (label[seed] >= 0) continue;
        // pseudo-peripheral node of this component
        int64_t root = seed;
        int last_depth = -1;
        for (int it = 0; it < 8; ++it) {
            std::vector<int32_t> q{(int32_t)root};
            std::vector<int32_t> seen{(int32_t)root};
            level[root] = 0;
            size_t h = 0;
            int depth = 0;
            while (h < q.size()) {
                int32_t u = q[h++];
                depth = std::max(depth, level[u]);
                for (int64_t p = aoff[u]; p < aoff[u + 1]; ++p)
                    if (level[adj[p]] < 0) { level[adj[p]] = level[u] + 1; q.push_back(adj[p]); seen.push_back(adj[p]); }
            }
            int64_t best = root;
            for (int32_t u : q)
                if (level[u] == depth && (deg(u) < deg(best) || level[best] != depth)) best = u;
            for (int32_t u : seen) level[u] = -1;
            if (depth <= last_depth) break;
            last_depth = depth;
            root = best;
        }
        // Cuthill-McKee breadth-first numbering, neighbours by increasing degree
        std::vector<int32_t> q{(int32_t)root};
        label[root] = next++;
        size_t h = 0;
        std::vector<int32_t> nb;
        while (h < q.size()) {
            int32_t u = q[h++];
            nb.clear();
            for (int64_t p = aoff[u]; p < aoff[u + 1]; ++p)
                if (label[adj[p]] < 0) nb.push_back(adj[p]);
            std::stable_sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) { return deg(a) < deg(b); });
            for (int32_t v : nb) { label[v] = next++; q.push_back(v); }
        }
    }
    std::vector<std::pair<int64_t, int32_t>> key(E);
    for (int64_t e = 0; e < E; ++e) {
        int64_t m = INT64_MAX;
        for (int k = 0; k < nv; ++k) m = std::min<int64_t>(m, (N - 1) - label[in.conn[e * nv + k]]);
        key[e] = {m, (int32_t)e};
    }
    std::sort(key.begin(), key.end());
    for (int64_t e = 0; e < E; ++e) elem_of[e] = key[e].second;
}

}  // namespace

std::string build_layout(const MeshInput& in, Layout& L, bool* mesh_error) {
    *mesh_error = false;
    const int nv = in.nv;
    const int64_t N = in.N, E = in.E;
    if ((int64_t)E * nv + 1 >= INT32_MAX) return "mesh too large for 32-bit slot ids";
    for (int64_t i = 0; i < E * nv; ++i)
        if (in.conn[i] < 0 || in.conn[i] >= N) {
            *mesh_error = true;
            return "element " + std::to_string(i / nv) + " references node " + std::to_string(in.conn[i]) +
                   " outside [0, n_nodes)";
        }
    L = Layout();
    L.nv = nv; L.N = N; L.E = E;
    L.elem_of.resize(E);
    if (in.order == FEDFEM_ORDER_MORTON) morton_order(in, L.elem_of);
    else if (in.order == FEDFEM_ORDER_RCM) rcm_order(in, L.elem_of);
    else std::iota(L.elem_of.begin(), L.elem_of.end(), 0);
    group_sort(in, L.elem_of);
    std::vector<int32_t> elem_at(E);
    for (int64_t e = 0; e < E; ++e) elem_at[L.elem_of[e]] = (int32_t)e;

    // first touch in the internal element order
    std::vector<int64_t> touch(N, -1);
    int64_t cnt = 0;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* c = in.conn + (int64_t)L.elem_of[e] * nv;
        for (int k = 0; k < nv; ++k)
            if (touch[c[k]] < 0) touch[c[k]] = cnt++;
    }
    if (cnt != N) {
        for (int64_t n = 0; n < N; ++n)
            if (touch[n] < 0) { *mesh_error = true; return "node " + std::to_string(n) + " is used by no element"; }
    }
    // classes: 0 plain free, 1 film (free), 2 Dirichlet
    std::vector<char> cls(N, 0);
    if (in.conv_faces)
        for (int32_t n : *in.conv_faces) cls[n] = 1;
    if (in.is_dirichlet)
        for (int64_t n = 0; n < N; ++n)
            if ((*in.is_dirichlet)[n]) cls[n] = 2;
    std::vector<int32_t> by_touch(N);
    for (int64_t n = 0; n < N; ++n) by_touch[touch[n]] = (int32_t)n;
    L.node_of.clear();
    L.node_of.reserve(N);
    for (int c = 0; c < 3; ++c) {
        for (int64_t t = 0; t < N; ++t)
            if (cls[by_touch[t]] == c) L.node_of.push_back(by_touch[t]);
        if (c == 0) L.N_plain = (int64_t)L.node_of.size();
        if (c == 1) L.N_free = (int64_t)L.node_of.size();
    }
    L.node_at.assign(N, 0);
    for (int64_t i = 0; i < N; ++i) L.node_at[L.node_of[i]] = (int32_t)i;
    L.conn.resize(E * nv);
    for (int64_t e = 0; e < E; ++e)
        for (int k = 0; k < nv; ++k)
            L.conn[e * nv + k] = L.node_at[in.conn[(int64_t)L.elem_of[e] * nv + k]];

    // node -> slot lists over free nodes, filled in INPUT element order
    const int64_t NF = L.N_free;
    std::vector<int64_t> off(NF + 1, 0);
    for (int64_t i = 0; i < E * nv; ++i) {
        int32_t n = L.node_at[in.conn[i]];
        if (n < NF) off[n + 1]++;
    }
    int maxdeg = 0;
    for (int64_t n = 0; n < NF; ++n) maxdeg = std::max<int>(maxdeg, (int)off[n + 1]);
    for (int64_t n = 0; n < NF; ++n) off[n + 1] += off[n];
    std::vector<int32_t> lists(off[NF]);
    {
        std::vector<int64_t> pos(off.begin(), off.end() - 1);
        for (int64_t ein = 0; ein < E; ++ein)
            for (int k = 0; k < nv; ++k) {
                int32_t n = L.node_at[in.conn[ein * nv + k]];
                if (n < NF) lists[pos[n]++] = elem_at[ein] * nv + k;
            }
    }
    L.max_degree = maxdeg;
    const int64_t n_slices = (NF + 31) / 32;
    L.sell_off.assign(n_slices + 1, 0);
    for (int64_t s = 0; s < n_slices; ++s) {
        int w = 0;
        for (int64_t n = 32 * s; n < std::min(NF, 32 * s + 32); ++n) w = std::max<int>(w, (int)(off[n + 1] - off[n]));
        if ((int64_t)L.sell_off[s] + 32LL * w >= INT32_MAX) return "gather structure too large for 32-bit offsets";
        L.sell_off[s + 1] = L.sell_off[s] + 32 * w;
    }
    const int32_t pad = (int32_t)(E * nv);
    L.sell_ids.assign(L.sell_off[n_slices], pad);
    for (int64_t n = 0; n < NF; ++n) {
        const int64_t s = n / 32, lane = n % 32;
        for (int64_t p = off[n]; p < off[n + 1]; ++p)
            L.sell_ids[L.sell_off[s] + 32 * (p - off[n]) + lane] = lists[p];
    }

    // film nodes -> faces (input face order)
    const int64_t NC = L.N_free - L.N_plain;
    L.conv_off.assign(NC + 1, 0);
    L.conv_face.clear();
    if (in.conv_faces && NC > 0) {
        const int fv = in.conv_nverts;
        const int64_t nf = (int64_t)in.conv_faces->size() / fv;
        std::vector<std::vector<int32_t>> per(NC);
        for (int64_t f = 0; f < nf; ++f)
            for (int k = 0; k < fv; ++k) {
                int32_t n = L.node_at[(*in.conv_faces)[f * fv + k]];
                if (n >= L.N_plain && n < L.N_free) {
                    auto& v = per[n - L.N_plain];
                    if (v.empty() || v.back() != (int32_t)f) v.push_back((int32_t)f);
                }
            }
        for (int64_t i = 0; i < NC; ++i) {
            L.conv_off[i + 1] = L.conv_off[i] + (int32_t)per[i].size();
            L.conv_face.insert(L.conv_face.end(), per[i].begin(), per[i].end());
        }
    }
    return "";
}

}  // namespace fedfem

namespace fedfem {

// Order of one tet tile's elements for the warps of the tiled kernels (each
// run of 32 consecutive elements is one warp): warp by warp, the next element
// is the one, among the first K not yet placed, that adds the fewest
// shared-memory bank collisions to the warp's accesses, corner by corner:
// temperature loads at the local id, load stores at rank x (B + 1) + id for
// owned corners.  Sums are taken in rank order, so the order changes no
// result.  lid, rnk: nv entries per element in the tile's sorted order.
static void bank_order(const std::vector<int32_t>& lid, const std::vector<uint8_t>& rnk, int nv, int64_t ne,
                       int64_t own, int64_t B, std::vector<int32_t>& perm) {
    constexpr int K = 48;
    perm.clear();
    // each corner's load word and store word (-1: a halo corner, no store), computed once
    std::vector<int32_t> lw(ne * nv), sw(ne * nv);
    for (int64_t q = 0; q < ne * nv; ++q) {
        lw[q] = lid[q];
        sw[q] = lid[q] < own ? (int32_t)(rnk[q] * (B + 1) + lid[q]) : -1;
    }
    // doubly linked list of the unplaced elements in sorted order; index ne is the sentinel
    std::vector<int32_t> nxt(ne + 1), prv(ne + 1);
    for (int64_t j = 0; j <= ne; ++j) {
        nxt[j] = (int32_t)((j + 1) % (ne + 1));
        prv[j] = (int32_t)((j + ne) % (ne + 1));
    }
    // the first word that took each bank in the warp being filled, per corner (-1: free)
    std::vector<int32_t> la(nv * 32), sa(nv * 32);
    for (int64_t placed = 0; placed < ne;) {
        std::fill(la.begin(), la.end(), -1);
        std::fill(sa.begin(), sa.end(), -1);
        for (int slot = 0; slot < 32 && placed < ne; ++slot, ++placed) {
            int32_t best = -1;
            int best_cost = 1 << 30;
            int seen = 0;
            for (int32_t j = nxt[ne]; j != ne && seen < K; j = nxt[j], ++seen) {
                const int32_t* l = &lw[(int64_t)j * nv];
                const int32_t* w = &sw[(int64_t)j * nv];
                int cost = 0;
                for (int k = 0; k < nv; ++k) {
                    const int32_t a = la[k * 32 + (l[k] & 31)];
                    cost += a >= 0 && a != l[k];
                    if (w[k] >= 0) {
                        const int32_t b = sa[k * 32 + (w[k] & 31)];
                        cost += b >= 0 && b != w[k];
                    }
                }
                if (cost < best_cost) {
                    best_cost = cost;
                    best = j;
                    if (cost == 0) break;
                }
            }
            perm.push_back(best);
            nxt[prv[best]] = nxt[best];
            prv[nxt[best]] = prv[best];
            const int32_t* l = &lw[(int64_t)best * nv];
            const int32_t* w = &sw[(int64_t)best * nv];
            for (int k = 0; k < nv; ++k) {
                if (la[k * 32 + (l[k] & 31)] < 0) la[k * 32 + (l[k] & 31)] = l[k];
                if (w[k] >= 0 && sa[k * 32 + (w[k] & 31)] < 0) sa[k * 32 + (w[k] & 31)] = w[k];
            }
        }
    }
}

std::string build_tiles(const Layout& L, int B, Tiles& T) {
    T = Tiles();
    const int nv = L.nv;
    const int64_t NF = L.N_free;
    if (B <= 0 || B % 8) return "tile size must be a positive multiple of 8";
    T.B = B; T.nv = nv;
    T.n_tiles = (NF + B - 1) / B;
    T.e_off.assign(T.n_tiles + 1, 0);
    T.h_off.assign(T.n_tiles + 1, 0);
    T.deg.assign(T.n_tiles, 0);
    std::vector<int32_t> elems, local_of(L.N, -1), rank_of;
    std::vector<int32_t> touched;
    std::vector<int32_t> lid;                      // local ids, combined with the ranks at the end
    std::vector<uint8_t> rank;
    std::vector<int32_t> tl, perm;                 // one tile: local ids (sorted element order), warp order
    std::vector<uint8_t> tr;
    for (int64_t t = 0; t < T.n_tiles; ++t) {
        const int64_t base = t * B, own = std::min<int64_t>(B, NF - base);
        // elements touching the owned nodes, from the nodes' slot lists
        elems.clear();
        for (int64_t i = base; i < base + own; ++i) {
            const int64_t s = i / 32, lane = i % 32;
            const int w = (L.sell_off[s + 1] - L.sell_off[s]) / 32;
            for (int k = 0; k < w; ++k) {
                const int32_t slot = L.sell_ids[L.sell_off[s] + 32 * k + lane];
                if (slot < L.E * nv) elems.push_back(slot / nv);
            }
        }
        std::sort(elems.begin(), elems.end());
        elems.erase(std::unique(elems.begin(), elems.end()), elems.end());
        const int64_t ne = (int64_t)elems.size();
        // local numbering: owned first, then halo in global order
        touched.clear();
        for (int32_t e : elems)
            for (int k = 0; k < nv; ++k) {
                const int32_t g = L.conn[(int64_t)e * nv + k];
                if (g < base || g >= base + own) touched.push_back(g);
            }
        std::sort(touched.begin(), touched.end());
        touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
        const int64_t nl = own + (int64_t)touched.size();
        if (nl > 65535) return "tile has too many local nodes for 16-bit ids; use smaller tiles";
        for (int64_t l = 0; l < own; ++l) local_of[base + l] = (int32_t)l;
        for (size_t h = 0; h < touched.size(); ++h) local_of[touched[h]] = (int32_t)(own + h);
        // rank of each (element, owned corner) in the corner node's slot list,
        // which is in input element order: the position its load takes in the sum
        rank_of.assign(ne * nv, 0);
        int dmax = 0;
        for (int64_t i = base; i < base + own; ++i) {
            const int64_t s = i / 32, lane = i % 32;
            const int w = (L.sell_off[s + 1] - L.sell_off[s]) / 32;
            int k = 0;
            for (; k < w; ++k) {
                const int32_t slot = L.sell_ids[L.sell_off[s] + 32 * k + lane];
                if (slot >= L.E * nv) break;                 // pads come last
                const int64_t j = std::lower_bound(elems.begin(), elems.end(), slot / nv) - elems.begin();
                rank_of[j * nv + slot % nv] = k;
            }
            dmax = std::max(dmax, k);
        }
        if (dmax > 255) return "a node has more than 255 elements";
        T.deg[t] = dmax;
        tl.resize(ne * nv);
        tr.resize(ne * nv);
        for (int64_t j = 0; j < ne; ++j)
            for (int k = 0; k < nv; ++k) {
                const int32_t l = local_of[L.conn[(int64_t)elems[j] * nv + k]];
                tl[j * nv + k] = l;
                tr[j * nv + k] = (uint8_t)(l < own ? rank_of[j * nv + k] : 0);
            }
        if (nv == 4) {
            bank_order(tl, tr, nv, ne, own, B, perm);
        } else {
            perm.resize(ne);
            for (int64_t j = 0; j < ne; ++j) perm[j] = (int32_t)j;
        }
        for (int64_t q = 0; q < ne; ++q) {
            const int64_t j = perm[q];
            T.e_glob.push_back(elems[j]);
            for (int k = 0; k < nv; ++k) {
                lid.push_back(tl[j * nv + k]);
                rank.push_back(tr[j * nv + k]);
            }
        }
        T.halo.insert(T.halo.end(), touched.begin(), touched.end());
        for (int64_t l = 0; l < own; ++l) local_of[base + l] = -1;
        for (int32_t g : touched) local_of[g] = -1;
        T.e_off[t + 1] = T.e_off[t] + (int32_t)ne;
        T.h_off[t + 1] = T.h_off[t] + (int32_t)touched.size();
        T.max_local = std::max<int>(T.max_local, (int)nl);
        T.max_elems = std::max<int>(T.max_elems, (int)ne);
        T.max_deg = std::max<int>(T.max_deg, dmax);
    }
    // 16-bit entries: local id in the low bits, rank above it
    int rank_bits = 0;
    while ((1 << rank_bits) < T.max_deg) ++rank_bits;
    T.rank_shift = 16 - rank_bits;
    if (T.max_local > (1 << T.rank_shift))
        return "tile has too many local nodes for its 16-bit ids and ranks; use smaller tiles";
    T.lconn.resize(lid.size());
    for (size_t q = 0; q < lid.size(); ++q)
        T.lconn[q] = (uint16_t)(lid[q] | (rank_bits ? (int)rank[q] << T.rank_shift : 0));
    return "";
}

}  // namespace fedfem
