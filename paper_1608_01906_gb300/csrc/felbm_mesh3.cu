// Host-side preprocessing of tetrahedral meshes (the paper's own 3-D
// setting): validation, P1 element geometry, lumped mass, assembled
// streaming / recovery coefficients and reverse Cuthill-McKee order.
//
// Sec. 2.2.1: with the lumped mass m_i = sum_{T∋i} |T|/4 the P1 streaming of
// a population with velocity e is
//   psi*_i = psi_i - dt sum_{j != i} (e.a_ij + dt/2 e.b_ij.e) (psi_j - psi_i),
//   a_ij = sum_{T∋i,j} |T| grad N_j / (4 m_i),
//   b_ij = sum_{T∋i,j} |T| / m_i grad N_i (x) grad N_j  (symmetric part),
// the difference form following from sum_j grad N_j = 0 on every element.
// Sec. 2.3: the volume-weighted recovery of a gradient is sum_j a_ij
// (f_j - f_i), the same a_ij (sum_{T∋i} |T| = 4 m_i).
#include <algorithm>
#include <cmath>

#include "felbm_internal.h"

namespace felbm {

static inline double wrap3(double d, double L) {
    if (L > 0.0) d -= L * std::nearbyint(d / L);
    return d;
}

struct Tet {
    double vol;
    double g[4][3];  // grad N_a of the four vertices
};

// Volume and shape-function gradients; vertices 1..3 at the minimum image of
// vertex 0.  grad N_{b+1} is column b of the inverse edge matrix, grad N_0
// minus their sum.  False for a non-positive volume.
static bool tet_geom(const double *xyz, const int32_t *v, const double L[3], Tet &t) {
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = wrap3(xyz[3 * v[r + 1] + c] - xyz[3 * v[0] + c], L[c]);
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det > 0.0) || !std::isfinite(det)) return false;
    const double inv[3][3] = {
        {c00 / det, (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det, (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det},
        {c01 / det, (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det, (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det},
        {c02 / det, (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det, (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det}};
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int b = 0; b < 3; ++b) {
            t.g[b + 1][c] = inv[c][b];
            s += inv[c][b];
        }
        t.g[0][c] = -s;
    }
    t.vol = det / 6.0;
    return true;
}

struct Entry3 {
    int32_t i, j;
    double c[9];  // ax, ay, az, bxx, bxy, bxz, byy, byz, bzz
};

int build_csr3(const double *xyz, int64_t n_nodes, const int32_t *tet, int64_t n_tet,
               const double box[3], uint32_t flags, const uint8_t *tag, HostCSR3 &out) {
    const int32_t N = (int32_t)n_nodes;
    const uint32_t pf[3] = {FELBM_PERIODIC_X, FELBM_PERIODIC_Y, FELBM_PERIODIC_Z};
    double L[3];
    for (int c = 0; c < 3; ++c) {
        L[c] = (flags & pf[c]) ? box[c] : 0.0;
        if ((flags & pf[c]) && !(box[c] > 0.0)) return FELBM_ERR_INVALID_ARG;
    }
    for (int64_t k = 0; k < 3 * n_nodes; ++k)
        if (!std::isfinite(xyz[k])) return FELBM_ERR_INVALID_MESH;
    if (tag)
        for (int64_t i = 0; i < n_nodes; ++i)
            if (tag[i] > 18) return FELBM_ERR_INVALID_MESH;
    std::vector<Tet> geo((size_t)n_tet);
    std::vector<double> mass((size_t)N, 0.0);
    for (int64_t t = 0; t < n_tet; ++t) {
        const int32_t *v = tet + 4 * t;
        for (int k = 0; k < 4; ++k)
            if (v[k] < 0 || v[k] >= N) return FELBM_ERR_INVALID_MESH;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (v[a] == v[b]) return FELBM_ERR_INVALID_MESH;
        if (!tet_geom(xyz, v, L, geo[t])) return FELBM_ERR_INVALID_MESH;
        for (int k = 0; k < 4; ++k) mass[v[k]] += geo[t].vol / 4.0;
    }
    for (int32_t i = 0; i < N; ++i)
        if (!(mass[i] > 0.0)) return FELBM_ERR_INVALID_MESH;
    std::vector<Entry3> ent;
    ent.reserve((size_t)n_tet * 12);
    for (int64_t t = 0; t < n_tet; ++t) {
        const int32_t *v = tet + 4 * t;
        const Tet &g = geo[t];
        for (int a = 0; a < 4; ++a) {
            const double mi = mass[v[a]];
            const double s = g.vol / mi;
            const double *gi = g.g[a];
            for (int b = 0; b < 4; ++b) {
                if (a == b) continue;
                const double *gj = g.g[b];
                Entry3 e;
                e.i = v[a];
                e.j = v[b];
                for (int c = 0; c < 3; ++c) e.c[c] = g.vol * gj[c] / (4.0 * mi);
                e.c[3] = s * gi[0] * gj[0];
                e.c[4] = s * 0.5 * (gi[0] * gj[1] + gi[1] * gj[0]);
                e.c[5] = s * 0.5 * (gi[0] * gj[2] + gi[2] * gj[0]);
                e.c[6] = s * gi[1] * gj[1];
                e.c[7] = s * 0.5 * (gi[1] * gj[2] + gi[2] * gj[1]);
                e.c[8] = s * gi[2] * gj[2];
                ent.push_back(e);
            }
        }
    }
    std::sort(ent.begin(), ent.end(), [](const Entry3 &p, const Entry3 &q) {
        return p.i != q.i ? p.i < q.i : p.j < q.j;
    });
    std::vector<Entry3> m;
    m.reserve(ent.size() / 4 + 8);
    for (const Entry3 &e : ent) {
        if (!m.empty() && m.back().i == e.i && m.back().j == e.j) {
            for (int k = 0; k < 9; ++k) m.back().c[k] += e.c[k];
        } else {
            m.push_back(e);
        }
    }
    ent.clear();
    ent.shrink_to_fit();
    std::vector<int32_t> rp0((size_t)N + 1, 0), cl0(m.size());
    for (const Entry3 &e : m) rp0[e.i + 1]++;
    for (int32_t i = 0; i < N; ++i) rp0[i + 1] += rp0[i];
    for (size_t k = 0; k < m.size(); ++k) cl0[k] = m[k].j;
    std::vector<int32_t> order = rcm_order(N, rp0, cl0);
    out.n = N;
    out.perm = order;
    out.iperm.assign((size_t)N, 0);
    for (int32_t k = 0; k < N; ++k) out.iperm[order[k]] = k;
    out.rowptr.assign((size_t)N + 1, 0);
    for (int32_t k = 0; k < N; ++k)
        out.rowptr[k + 1] = out.rowptr[k] + (rp0[order[k] + 1] - rp0[order[k]]);
    const size_t nnz = m.size();
    out.col.resize(nnz);
    out.coef.assign(9 * nnz, 0.0);
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int32_t k = 0; k < N; ++k) {
        const int32_t old = order[k];
        row.clear();
        for (int32_t p = rp0[old]; p < rp0[old + 1]; ++p) row.push_back({out.iperm[cl0[p]], p});
        std::sort(row.begin(), row.end());
        int32_t q = out.rowptr[k];
        for (auto &rc : row) {
            out.col[q] = rc.first;
            for (int c = 0; c < 9; ++c) out.coef[(size_t)c * nnz + q] = m[rc.second].c[c];
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

}  // namespace felbm

namespace felbm {

static int offset_index3(int dx, int dy, int dz) {
    for (int o = 0; o < 14; ++o)
        if (lat3_dx(o) == dx && lat3_dy(o) == dy && lat3_dz(o) == dz) return o;
    return -1;
}

// The mesh is the Kuhn lattice when the nodes sit on an (nx, ny, nz) grid in
// id order, the flags and tags are those of structured_tet_mesh (periodic x
// and y, z periodic or walled by tags 5 and 6), every node's neighbours are
// the 14 lattice offsets and every node's assembled coefficients equal those
// of the first node of its z-layer kind (to 1e-12 of the largest).
void detect_lattice3(const double *xyz, int64_t n_nodes, const double box[3], uint32_t flags,
                     const uint8_t *tag, const HostCSR3 &H, Lattice3Info &info) {
    info.ok = false;
    if (!(flags & FELBM_PERIODIC_X) || !(flags & FELBM_PERIODIC_Y) || n_nodes < 27) return;
    const double h = xyz[3] - xyz[0];
    if (!(h > 0.0)) return;
    int64_t nx = 0;
    while (nx < n_nodes && std::fabs(xyz[3 * nx + 1] - xyz[1]) <= 1e-12 * h &&
           std::fabs(xyz[3 * nx + 2] - xyz[2]) <= 1e-12 * h)
        ++nx;
    int64_t layer = 0;
    while (layer < n_nodes && std::fabs(xyz[3 * layer + 2] - xyz[2]) <= 1e-12 * h) ++layer;
    if (nx < 3 || layer % nx || n_nodes % layer) return;
    const int64_t ny = layer / nx, nz = n_nodes / layer;
    if (ny < 3 || nz < 3 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return;
    const double tol = 1e-9 * h;
    for (int64_t i = 0; i < n_nodes; ++i) {
        const int64_t x = i % nx, y = (i / nx) % ny, z = i / layer;
        if (std::fabs(xyz[3 * i] - (xyz[0] + x * h)) > tol || std::fabs(xyz[3 * i + 1] - (xyz[1] + y * h)) > tol ||
            std::fabs(xyz[3 * i + 2] - (xyz[2] + z * h)) > tol)
            return;
    }
    if (std::fabs(box[0] - nx * h) > tol || std::fabs(box[1] - ny * h) > tol) return;
    const bool pz = (flags & FELBM_PERIODIC_Z) != 0;
    if (pz && std::fabs(box[2] - nz * h) > tol) return;
    if (!pz) {
        if (!tag) return;
        for (int64_t i = 0; i < n_nodes; ++i) {
            const int64_t z = i / layer;
            if (tag[i] != (z == 0 ? 5 : (z == nz - 1 ? 6 : 0))) return;
        }
    } else if (tag) {
        for (int64_t i = 0; i < n_nodes; ++i)
            if (tag[i]) return;
    }
    bool have[3] = {false, false, false};
    int count[3] = {0, 0, 0};
    double c[3][14][9] = {};
    double cmax = 0.0;
    for (double v : H.coef) cmax = std::max(cmax, std::fabs(v));
    const size_t nnz = H.col.size();
    for (int32_t k = 0; k < H.n; ++k) {
        const int64_t ci = H.perm[k];
        const int64_t x = ci % nx, y = (ci / nx) % ny, z = ci / layer;
        const int kind = pz ? 0 : (z == 0 ? 1 : (z == nz - 1 ? 2 : 0));
        const int deg = H.rowptr[k + 1] - H.rowptr[k];
        double row[14][9] = {};
        bool seen[14] = {};
        for (int32_t p = H.rowptr[k]; p < H.rowptr[k + 1]; ++p) {
            const int64_t cj = H.perm[H.col[p]];
            int64_t dx = cj % nx - x, dy = (cj / nx) % ny - y, dz = cj / layer - z;
            if (dx > 1) dx -= nx;
            if (dx < -1) dx += nx;
            if (dy > 1) dy -= ny;
            if (dy < -1) dy += ny;
            if (pz && dz > 1) dz -= nz;
            if (pz && dz < -1) dz += nz;
            const int o = offset_index3((int)dx, (int)dy, (int)dz);
            if (o < 0 || seen[o]) return;
            seen[o] = true;
            for (int q = 0; q < 9; ++q) row[o][q] = H.coef[(size_t)q * nnz + p];
        }
        if (!have[kind]) {
            have[kind] = true;
            count[kind] = deg;
            for (int o = 0; o < 14; ++o)
                for (int q = 0; q < 9; ++q) c[kind][o][q] = row[o][q];
        } else {
            if (deg != count[kind]) return;
            for (int o = 0; o < 14; ++o)
                for (int q = 0; q < 9; ++q)
                    if (std::fabs(row[o][q] - c[kind][o][q]) > 1e-12 * cmax) return;
        }
    }
    info.nx = (int32_t)nx;
    info.ny = (int32_t)ny;
    info.nz = (int32_t)nz;
    info.walls = !pz;
    for (int k = 0; k < 3; ++k)
        for (int o = 0; o < 14; ++o)
            for (int q = 0; q < 9; ++q) info.c[k][o][q] = c[k][o][q];
    info.ok = true;
}

}  // namespace felbm
