// Host-side mesh preprocessing: validation, P1 element geometry, lumped mass,
// assembled streaming / recovery coefficients, reverse Cuthill-McKee order,
// and recognition of the structured lattice split.
//
// Geometry and operators follow Sec. 2.2.1 (P1 Bubnov-Galerkin form of the
// Taylor-expanded streaming with the lumped mass matrix) and Sec. 2.3
// (element gradients averaged with element-area weights).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>

#include "felbm_internal.h"

namespace felbm {

static inline double wrap(double d, double L) {
    if (L > 0.0) d -= L * std::nearbyint(d / L);
    return d;
}

struct ElemGeom {
    double area;
    double gx[3], gy[3];  // grad N_a for the three vertices
};

// Element area and shape-function gradients with the second and third vertex
// taken at the minimum image of the first.  Returns false for area <= 0.
static bool elem_geom(const double *xy, const int32_t *t, const double Lp[2], ElemGeom &g) {
    const int32_t a = t[0], b = t[1], c = t[2];
    const double xb = wrap(xy[2 * b] - xy[2 * a], Lp[0]);
    const double yb = wrap(xy[2 * b + 1] - xy[2 * a + 1], Lp[1]);
    const double xc = wrap(xy[2 * c] - xy[2 * a], Lp[0]);
    const double yc = wrap(xy[2 * c + 1] - xy[2 * a + 1], Lp[1]);
    const double det = xb * yc - xc * yb;  // 2 |T|
    if (!(det > 0.0) || !std::isfinite(det)) return false;
    const double inv = 1.0 / det;
    g.area = 0.5 * det;
    g.gx[0] = (yb - yc) * inv;  g.gy[0] = (xc - xb) * inv;
    g.gx[1] = (yc - 0.0) * inv; g.gy[1] = (0.0 - xc) * inv;
    g.gx[2] = (0.0 - yb) * inv; g.gy[2] = (xb - 0.0) * inv;
    return true;
}

struct Entry {
    int32_t i, j;
    double ax, ay, bxx, bxy, byy;
};

// Reverse Cuthill-McKee on the node graph given as CSR (rowptr/col, no
// self loops).  Every connected component is ordered from a pseudo-peripheral
// start node (lowest degree, then the farthest node of a BFS from it).
std::vector<int32_t> rcm_order(int32_t n, const std::vector<int32_t> &rp,
                               const std::vector<int32_t> &cl) {
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<char> seen(n, 0);
    std::vector<int32_t> deg(n);
    for (int32_t i = 0; i < n; ++i) deg[i] = rp[i + 1] - rp[i];
    std::vector<int32_t> by_deg(n);
    for (int32_t i = 0; i < n; ++i) by_deg[i] = i;
    std::stable_sort(by_deg.begin(), by_deg.end(),
                     [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
    std::vector<int32_t> level(n, -1);
    auto bfs_far = [&](int32_t s) {
        // farthest node from s within its component (ties: lowest degree)
        std::vector<int32_t> q{s};
        level[s] = 0;
        size_t h = 0;
        int32_t far = s;
        while (h < q.size()) {
            int32_t u = q[h++];
            if (level[u] > level[far] || (level[u] == level[far] && deg[u] < deg[far])) far = u;
            for (int32_t p = rp[u]; p < rp[u + 1]; ++p) {
                int32_t v = cl[p];
                if (level[v] < 0) {
                    level[v] = level[u] + 1;
                    q.push_back(v);
                }
            }
        }
        for (int32_t u : q) level[u] = -1;
        return far;
    };
    for (int32_t s0 : by_deg) {
        if (seen[s0]) continue;
        int32_t s = bfs_far(s0);
        size_t head = order.size();
        order.push_back(s);
        seen[s] = 1;
        std::vector<int32_t> nb;
        while (head < order.size()) {
            int32_t u = order[head++];
            nb.clear();
            for (int32_t p = rp[u]; p < rp[u + 1]; ++p)
                if (!seen[cl[p]]) nb.push_back(cl[p]);
            std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            for (int32_t v : nb) {
                seen[v] = 1;
                order.push_back(v);
            }
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// Conformity of a P1 triangulation (the Galerkin streaming of Sec. 2.2.1
// assumes a conforming mesh): every edge lies in at most two triangles, an
// edge of two triangles is traversed in opposite directions by them (both
// counter-clockwise), an edge of one triangle lies on the boundary of a
// non-periodic direction (both ends on the lowest or both on the highest
// coordinate of the nodes in that direction), and, with both directions
// periodic, the triangles tile the box once (areas sum to the box area).
static bool conforming(const double *xy, int32_t N, const int32_t *tri, int64_t n_tri, const double Lp[2],
                       const std::vector<ElemGeom> &geo) {
    std::vector<uint64_t> ed;  // (low end, high end, direction) per triangle side
    ed.reserve((size_t)n_tri * 3);
    for (int64_t t = 0; t < n_tri; ++t)
        for (int k = 0; k < 3; ++k) {
            const uint32_t a = (uint32_t)tri[3 * t + k], b = (uint32_t)tri[3 * t + (k + 1) % 3];
            const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
            ed.push_back((lo * (uint64_t)N + hi) << 1 | (a < b ? 0u : 1u));
        }
    std::sort(ed.begin(), ed.end());
    double lo[2] = {xy[0], xy[1]}, hi[2] = {xy[0], xy[1]};
    for (int32_t i = 1; i < N; ++i)
        for (int d = 0; d < 2; ++d) {
            lo[d] = std::min(lo[d], xy[2 * i + d]);
            hi[d] = std::max(hi[d], xy[2 * i + d]);
        }
    auto on_boundary = [&](uint32_t a, uint32_t b) {
        for (int d = 0; d < 2; ++d) {
            if (Lp[d] > 0.0) continue;
            const double tol = 1e-9 * std::max(hi[d] - lo[d], 1.0);
            if (std::fabs(xy[2 * a + d] - lo[d]) <= tol && std::fabs(xy[2 * b + d] - lo[d]) <= tol) return true;
            if (std::fabs(xy[2 * a + d] - hi[d]) <= tol && std::fabs(xy[2 * b + d] - hi[d]) <= tol) return true;
        }
        return false;
    };
    for (size_t k = 0; k < ed.size();) {
        size_t m = k + 1;
        while (m < ed.size() && (ed[m] >> 1) == (ed[k] >> 1)) ++m;
        const uint64_t key = ed[k] >> 1;
        if (m - k > 2) return false;
        if (m - k == 2 && (ed[k] & 1u) == (ed[k + 1] & 1u)) return false;
        if (m - k == 1 && !on_boundary((uint32_t)(key / (uint64_t)N), (uint32_t)(key % (uint64_t)N)))
            return false;
        k = m;
    }
    if (Lp[0] > 0.0 && Lp[1] > 0.0) {
        double area = 0.0;
        for (const ElemGeom &g : geo) area += g.area;
        if (std::fabs(area - Lp[0] * Lp[1]) > 1e-9 * Lp[0] * Lp[1]) return false;
    }
    return true;
}

int build_csr(const double *xy, int64_t n_nodes, const int32_t *tri, int64_t n_tri,
              const double box[2], uint32_t flags, const uint8_t *tag, HostCSR &out) {
    const int32_t N = (int32_t)n_nodes;
    const double Lp[2] = {(flags & FELBM_PERIODIC_X) ? box[0] : 0.0,
                          (flags & FELBM_PERIODIC_Y) ? box[1] : 0.0};
    if (((flags & FELBM_PERIODIC_X) && !(box[0] > 0.0)) ||
        ((flags & FELBM_PERIODIC_Y) && !(box[1] > 0.0)))
        return FELBM_ERR_INVALID_ARG;
    for (int64_t k = 0; k < 2 * n_nodes; ++k)
        if (!std::isfinite(xy[k])) return FELBM_ERR_INVALID_MESH;
    if (tag)
        for (int64_t i = 0; i < n_nodes; ++i)
            if (tag[i] > 8) return FELBM_ERR_INVALID_MESH;
    std::vector<ElemGeom> geo((size_t)n_tri);
    std::vector<double> mass((size_t)N, 0.0);
    for (int64_t t = 0; t < n_tri; ++t) {
        const int32_t *v = tri + 3 * t;
        for (int k = 0; k < 3; ++k)
            if (v[k] < 0 || v[k] >= N) return FELBM_ERR_INVALID_MESH;
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return FELBM_ERR_INVALID_MESH;
        if (!elem_geom(xy, v, Lp, geo[t])) return FELBM_ERR_INVALID_MESH;
        for (int k = 0; k < 3; ++k) mass[v[k]] += geo[t].area / 3.0;
    }
    for (int32_t i = 0; i < N; ++i)
        if (!(mass[i] > 0.0)) return FELBM_ERR_INVALID_MESH;  // isolated node
    if (!conforming(xy, N, tri, n_tri, Lp, geo)) return FELBM_ERR_INVALID_MESH;
    // assemble a_ij, b_ij (j != i) as triplets, then merge duplicates
    std::vector<Entry> ent;
    ent.reserve((size_t)n_tri * 6);
    for (int64_t t = 0; t < n_tri; ++t) {
        const int32_t *v = tri + 3 * t;
        const ElemGeom &g = geo[t];
        for (int a = 0; a < 3; ++a) {
            const double mi = mass[v[a]];
            for (int b = 0; b < 3; ++b) {
                if (a == b) continue;
                Entry e;
                e.i = v[a];
                e.j = v[b];
                e.ax = g.area * g.gx[b] / (3.0 * mi);
                e.ay = g.area * g.gy[b] / (3.0 * mi);
                const double s = g.area / mi;
                e.bxx = s * g.gx[a] * g.gx[b];
                e.byy = s * g.gy[a] * g.gy[b];
                e.bxy = s * 0.5 * (g.gx[a] * g.gy[b] + g.gy[a] * g.gx[b]);
                ent.push_back(e);
            }
        }
    }
    std::sort(ent.begin(), ent.end(), [](const Entry &p, const Entry &q) {
        return p.i != q.i ? p.i < q.i : p.j < q.j;
    });
    std::vector<Entry> m;
    m.reserve(ent.size() / 2 + 8);
    for (const Entry &e : ent) {
        if (!m.empty() && m.back().i == e.i && m.back().j == e.j) {
            Entry &b = m.back();
            b.ax += e.ax; b.ay += e.ay; b.bxx += e.bxx; b.bxy += e.bxy; b.byy += e.byy;
        } else {
            m.push_back(e);
        }
    }
    ent.clear();
    ent.shrink_to_fit();
    // graph in caller order for RCM
    std::vector<int32_t> rp0((size_t)N + 1, 0), cl0(m.size());
    for (const Entry &e : m) rp0[e.i + 1]++;
    for (int32_t i = 0; i < N; ++i) rp0[i + 1] += rp0[i];
    for (size_t k = 0; k < m.size(); ++k) cl0[k] = m[k].j;  // m sorted by (i, j)
    std::vector<int32_t> order = rcm_order(N, rp0, cl0);
    out.n = N;
    out.perm = order;
    out.iperm.assign((size_t)N, 0);
    for (int32_t k = 0; k < N; ++k) out.iperm[order[k]] = k;
    // CSR in internal order, columns sorted
    out.rowptr.assign((size_t)N + 1, 0);
    for (int32_t k = 0; k < N; ++k) out.rowptr[k + 1] = out.rowptr[k] + (rp0[order[k] + 1] - rp0[order[k]]);
    const size_t nnz = m.size();
    out.col.resize(nnz);
    out.ax.resize(nnz); out.ay.resize(nnz);
    out.bxx.resize(nnz); out.bxy.resize(nnz); out.byy.resize(nnz);
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int32_t k = 0; k < N; ++k) {
        const int32_t old = order[k];
        row.clear();
        for (int32_t p = rp0[old]; p < rp0[old + 1]; ++p) row.push_back({out.iperm[cl0[p]], p});
        std::sort(row.begin(), row.end());
        int32_t q = out.rowptr[k];
        for (auto &rc : row) {
            const Entry &e = m[rc.second];
            out.col[q] = rc.first;
            out.ax[q] = e.ax; out.ay[q] = e.ay;
            out.bxx[q] = e.bxx; out.bxy[q] = e.bxy; out.byy[q] = e.byy;
            ++q;
        }
    }
    out.mass.resize(N);
    for (int32_t k = 0; k < N; ++k) out.mass[k] = mass[order[k]];
    out.tag.clear();
    bool any_wall = false;
    if (tag)
        for (int32_t i = 0; i < N; ++i) any_wall |= tag[i] != 0;
    if (any_wall) {
        out.tag.resize(N);
        for (int32_t k = 0; k < N; ++k) out.tag[k] = tag[order[k]];
    }
    return FELBM_OK;
}

// A mesh is the structured lattice split when node i sits at
// ((i mod nx) h, (i div nx) h), every square (i, j) is cut along its
// (i,j)-(i+1,j+1) diagonal into [(i,j),(i+1,j),(i+1,j+1)] and
// [(i,j),(i+1,j+1),(i,j+1)] (any listing order / rotation), x is periodic with
// period nx h, and y is either periodic with period ny h or bounded with every
// node of row 0 tagged 2 and of row ny-1 tagged 4 and no other tag.
void detect_structured(const double *xy, int64_t n_nodes, const int32_t *tri, int64_t n_tri,
                       const double box[2], uint32_t flags, const uint8_t *tag,
                       StructuredInfo &info, std::vector<double> &mass) {
    info.ok = false;
    if (n_nodes < 16 || !(flags & FELBM_PERIODIC_X)) return;
    // nx from the first row: nodes with y == y0 in increasing x
    const double h = xy[2] - xy[0];
    if (!(h > 0.0)) return;
    int64_t nx = 0;
    while (nx < n_nodes && std::fabs(xy[2 * nx + 1] - xy[1]) <= 1e-12 * h) ++nx;
    if (nx < 4 || n_nodes % nx) return;
    const int64_t ny = n_nodes / nx;
    if (ny < 4 || nx > (1 << 20) || ny > (1 << 20)) return;
    const double tol = 1e-9 * h;
    for (int64_t i = 0; i < n_nodes; ++i) {
        const double ex = xy[0] + (double)(i % nx) * h, ey = xy[1] + (double)(i / nx) * h;
        if (std::fabs(xy[2 * i] - ex) > tol || std::fabs(xy[2 * i + 1] - ey) > tol) return;
    }
    if (std::fabs(box[0] - (double)nx * h) > tol) return;
    const bool py = (flags & FELBM_PERIODIC_Y) != 0;
    if (py && std::fabs(box[1] - (double)ny * h) > tol) return;
    bool walls = false;
    if (!py) {
        if (!tag) return;
        for (int64_t i = 0; i < n_nodes; ++i) {
            const int64_t j = i / nx;
            const uint8_t want = j == 0 ? 2 : (j == ny - 1 ? 4 : 0);
            if (tag[i] != want) return;
        }
        walls = true;
    } else if (tag) {
        for (int64_t i = 0; i < n_nodes; ++i)
            if (tag[i]) return;
    }
    const int64_t nsq_y = py ? ny : ny - 1;
    if (n_tri != 2 * nx * nsq_y) return;
    // every triangle must be one of the two canonical ones of its square;
    // count each square's two triangles exactly once.
    std::vector<uint8_t> have((size_t)(nx * nsq_y), 0);
    for (int64_t t = 0; t < n_tri; ++t) {
        int32_t v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        // rotate so that v[0] is the node whose (i, j) is the square's corner:
        bool matched = false;
        for (int r = 0; r < 3 && !matched; ++r) {
            const int32_t a = v[r], b = v[(r + 1) % 3], c = v[(r + 2) % 3];
            const int64_t ia = a % nx, ja = a / nx;
            const int64_t i1 = (ia + 1) % nx, j1 = (ja + 1) % ny;
            if (!py && ja + 1 >= ny) continue;
            const int64_t n_b = i1 + nx * ja, n_c = i1 + nx * j1, n_d = ia + nx * j1;
            const size_t sq = (size_t)(ia + nx * ja);
            if (b == n_b && c == n_c && !(have[sq] & 1)) { have[sq] |= 1; matched = true; }
            else if (b == n_c && c == n_d && !(have[sq] & 2)) { have[sq] |= 2; matched = true; }
        }
        if (!matched) return;
    }
    // Lumped mass of every node and, for a representative node of each row
    // kind (interior, bottom wall row, top wall row), the assembled a_ij,
    // b_ij of its six neighbours, from the triangles incident to it (the same
    // element formulas as the general assembly; every node of a kind has
    // the same coefficients by translation invariance).
    const double Lp[2] = {box[0], py ? box[1] : 0.0};
    static const int OFF[6][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 0}, {-1, -1}, {0, -1}};
    const int64_t rows[3] = {ny / 2, 0, ny - 1};
    int32_t rep[3];
    for (int kind = 0; kind < 3; ++kind) rep[kind] = (int32_t)(nx / 2 + nx * rows[kind]);
    mass.assign((size_t)n_nodes, 0.0);
    std::vector<ElemGeom> rep_geo[3];
    std::vector<int32_t> rep_tri[3];
    for (int64_t t = 0; t < n_tri; ++t) {
        ElemGeom g;
        if (!elem_geom(xy, tri + 3 * t, Lp, g)) return;
        for (int k = 0; k < 3; ++k) mass[tri[3 * t + k]] += g.area / 3.0;
        for (int kind = 0; kind < 3; ++kind)
            for (int k = 0; k < 3; ++k)
                if (tri[3 * t + k] == rep[kind]) {
                    rep_geo[kind].push_back(g);
                    rep_tri[kind].push_back((int32_t)t);
                }
    }
    for (int kind = 0; kind < 3; ++kind) {
        const int64_t j = rows[kind];
        const int64_t i = nx / 2;
        const int32_t node = rep[kind];
        const double mi = mass[node];
        for (int o = 0; o < 6; ++o) {
            info.a[kind][o][0] = info.a[kind][o][1] = 0.0;
            info.b[kind][o][0] = info.b[kind][o][1] = info.b[kind][o][2] = 0.0;
            const int64_t jj = j + OFF[o][1];
            if (!py && (jj < 0 || jj >= ny)) continue;
            const int32_t nb = (int32_t)(((i + OFF[o][0] + nx) % nx) + nx * ((jj + ny) % ny));
            for (size_t q = 0; q < rep_tri[kind].size(); ++q) {
                const int32_t *v = tri + 3 * rep_tri[kind][q];
                const ElemGeom &g = rep_geo[kind][q];
                int a = -1, b = -1;
                for (int k = 0; k < 3; ++k) {
                    if (v[k] == node) a = k;
                    if (v[k] == nb) b = k;
                }
                if (a < 0 || b < 0) continue;
                info.a[kind][o][0] += g.area * g.gx[b] / (3.0 * mi);
                info.a[kind][o][1] += g.area * g.gy[b] / (3.0 * mi);
                const double sc = g.area / mi;
                info.b[kind][o][0] += sc * g.gx[a] * g.gx[b];
                info.b[kind][o][1] += sc * 0.5 * (g.gx[a] * g.gy[b] + g.gy[a] * g.gx[b]);
                info.b[kind][o][2] += sc * g.gy[a] * g.gy[b];
            }
        }
    }
    info.nx = (int32_t)nx;
    info.pitch = (int32_t)((nx + 3) & ~(int64_t)3);
    info.ny = (int32_t)ny;
    info.walls = walls;
    info.h = h;
    info.row0 = info.ylo = 0;
    info.gny = info.yhi = (int32_t)ny;
    info.ok = true;
}

}  // namespace felbm
