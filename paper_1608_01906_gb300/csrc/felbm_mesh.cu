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

// Index of cell (x, y) along the Hilbert curve over a 2^k x 2^k grid (n =
// 2^k): descend through the quadrants, adding the cells of the quadrants the
// curve visits first, and turn the coordinates into the visited quadrant's
// own frame (Hilbert's construction, as in the usual iterative form).
static uint64_t hilbert_index(uint32_t n, uint32_t x, uint32_t y) {
    uint64_t d = 0;
    for (uint32_t s = n / 2; s > 0; s /= 2) {
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - (x & (s - 1));
                y = s - 1 - (y & (s - 1));
            } else {
                x &= s - 1;
                y &= s - 1;
            }
            const uint32_t t = x;
            x = y;
            y = t;
        } else {
            x &= s - 1;
            y &= s - 1;
        }
    }
    return d;
}

// Internal order of a general mesh: nodes sorted along a Hilbert curve over
// a grid about twice as fine as the node spacing, cut into patches of kPatch
// consecutive nodes (compact pieces of the mesh), each patch in the reverse
// Cuthill-McKee order of rcm (rcm[k] = caller id of RCM rank k).
static std::vector<int32_t> patch_order(const double *xy, int32_t N, const double Lp[2],
                                        const std::vector<int32_t> &rcm) {
    double lo[2] = {0, 0}, ext[2] = {0, 0};
    for (int d = 0; d < 2; ++d) {
        if (Lp[d] > 0.0) {
            ext[d] = Lp[d];
            continue;
        }
        double a = xy[d], b = xy[d];
        for (int32_t i = 1; i < N; ++i) {
            a = std::min(a, xy[2 * i + d]);
            b = std::max(b, xy[2 * i + d]);
        }
        lo[d] = a;
        ext[d] = std::max(b - a, 1e-300);
    }
    uint32_t n = 1;
    while ((double)n * n < 4.0 * N && n < (1u << 16)) n *= 2;
    const double cell = std::max(ext[0], ext[1]) / n;
    std::vector<int32_t> rank((size_t)N);
    for (int32_t k = 0; k < N; ++k) rank[rcm[k]] = k;
    std::vector<std::pair<uint64_t, int32_t>> key((size_t)N);
    for (int32_t i = 0; i < N; ++i) {
        uint32_t q[2];
        for (int d = 0; d < 2; ++d) {
            double v = xy[2 * i + d] - lo[d];
            if (Lp[d] > 0.0) v -= Lp[d] * std::floor(v / Lp[d]);
            const double c = std::floor(v / cell);
            q[d] = (uint32_t)std::min(std::max(c, 0.0), (double)(n - 1));
        }
        key[i] = {hilbert_index(n, q[0], q[1]), rank[i]};
    }
    std::vector<int32_t> order((size_t)N);
    for (int32_t i = 0; i < N; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    for (int32_t p0 = 0; p0 < N; p0 += kPatch) {
        const int32_t p1 = std::min(N, p0 + kPatch);
        std::sort(order.begin() + p0, order.begin() + p1,
                  [&](int32_t a, int32_t b) { return rank[a] < rank[b]; });
    }
    return order;
}

// Rings of every patch over the CSR in internal (patch-major) order.
static void build_patches(HostCSR &H) {
    const int32_t N = H.n, np = (N + kPatch - 1) / kPatch;
    H.pnbase.assign((size_t)np + 1, 0);
    H.pcount.assign((size_t)4 * np, 0);
    H.pnode.clear();
    H.prowbase.clear();
    H.plcol.clear();
    H.rmax = H.r1max = H.r2max = H.r3max = 0;
    std::vector<int32_t> stamp((size_t)N, -1), loc((size_t)N, 0);
    std::vector<int32_t> reg;
    for (int32_t p = 0; p < np; ++p) {
        reg.clear();
        for (int32_t i = p * kPatch; i < std::min(N, (p + 1) * kPatch); ++i) {
            stamp[i] = p;
            loc[i] = (int32_t)reg.size();
            reg.push_back(i);
        }
        int32_t cnt[4];
        size_t ring0 = 0;
        for (int ring = 1; ring <= 4; ++ring) {
            cnt[ring - 1] = (int32_t)reg.size();
            const size_t ring1 = reg.size();
            for (size_t k = ring0; k < ring1; ++k)
                for (int32_t e = H.rowptr[reg[k]]; e < H.rowptr[reg[k] + 1]; ++e) {
                    const int32_t j = H.col[e];
                    if (stamp[j] != p) {
                        stamp[j] = p;
                        loc[j] = (int32_t)reg.size();
                        reg.push_back(j);
                    }
                }
            ring0 = ring1;
        }
        if (reg.size() > 65535) {  // region indices are 16-bit: no patch step
            H.pnbase.clear();
            H.pcount.clear();
            H.pnode.clear();
            H.prowbase.clear();
            H.plcol.clear();
            return;
        }
        for (int r = 0; r < 4; ++r) H.pcount[4 * p + r] = cnt[r];
        H.pnbase[p + 1] = H.pnbase[p] + (int32_t)reg.size();
        for (size_t r = 0; r < reg.size(); ++r) {
            H.pnode.push_back(reg[r]);
            if ((int32_t)r < cnt[3]) {
                H.prowbase.push_back((int32_t)H.plcol.size());
                for (int32_t e = H.rowptr[reg[r]]; e < H.rowptr[reg[r] + 1]; ++e)
                    H.plcol.push_back((uint16_t)loc[H.col[e]]);
            } else {
                H.prowbase.push_back(-1);
            }
        }
        H.rmax = std::max(H.rmax, (int32_t)reg.size());
        H.r1max = std::max(H.r1max, cnt[1]);
        H.r2max = std::max(H.r2max, cnt[2]);
        H.r3max = std::max(H.r3max, cnt[3]);
    }
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
    std::vector<int32_t> order = patch_order(xy, N, Lp, rcm_order(N, rp0, cl0));
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
    build_patches(out);
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
