// Host-side tearing of the mesh (Sec. III-A) and Whitney element matrices (Sec. II-B).
//
// Everything here runs once per dd_setup on the CPU: edge extraction and
// orientation, PEC edge removal, per-tet mass/curl-curl matrices, edge
// multiplicities, local numbering [interior | interface | corner], the signed
// Boolean B_r (one multiplier per edge shared by two subdomains, +1 in the lower
// subdomain id) and the unsigned Boolean B_c (corners = edges shared by three or
// more subdomains), and the subassembled local CSR matrices.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "dd_internal.h"

namespace {

// local edge k of a tet joins local vertices kEdge[k][0] -> kEdge[k][1]
const int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const int kFace[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

inline void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Tangential Whitney mass of a triangle (nodes p[0..2], ids increasing) over its
// edges (0,1), (1,2), (0,2), each oriented low -> high: the tangential trace of
// a 3-D Whitney function is the 2-D one l_a g_b - l_b g_a (g: surface gradients
// of the triangle's barycentrics, g_k = sum_j (G^-1)_kj E_j with E_j = p_j - p_0,
// G the 2x2 metric), integrated with int l_a l_c = area (1 + delta_ac) / 12.
void face_mass(const double* p0, const double* p1, const double* p2, double M[9]) {
    double E1[3], E2[3];
    for (int c = 0; c < 3; ++c) {
        E1[c] = p1[c] - p0[c];
        E2[c] = p2[c] - p0[c];
    }
    const double g11 = dot3(E1, E1), g12 = dot3(E1, E2), g22 = dot3(E2, E2);
    const double det = g11 * g22 - g12 * g12;
    const double i11 = g22 / det, i12 = -g12 / det, i22 = g11 / det;
    double g[3][3];
    for (int c = 0; c < 3; ++c) {
        g[1][c] = i11 * E1[c] + i12 * E2[c];
        g[2][c] = i12 * E1[c] + i22 * E2[c];
        g[0][c] = -g[1][c] - g[2][c];
    }
    const double area = 0.5 * std::sqrt(det);
    double gg[3][3], ll[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            gg[a][b] = dot3(g[a], g[b]);
            ll[a][b] = area * (a == b ? 2.0 : 1.0) / 12.0;
        }
    const int fe[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            const int a = fe[p][0], b = fe[p][1], c = fe[q][0], d = fe[q][1];
            M[3 * p + q] = ll[a][c] * gg[b][d] - ll[a][d] * gg[b][c] - ll[b][c] * gg[a][d] + ll[b][d] * gg[a][c];
        }
}

// Barycentric gradients g[4][3] and |volume| of a tet.  With d_i = X_i - X_0 and
// det = d1 . (d2 x d3): grad l1 = d2 x d3 / det, grad l2 = d3 x d1 / det,
// grad l3 = d1 x d2 / det, grad l0 = -(sum).  Returns the signed det.
double tet_gradients(const double* X, double g[4][3], double* volume) {
    double d[3][3];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) d[i][c] = X[3 * (i + 1) + c] - X[c];
    double c23[3], c31[3], c12[3];
    cross3(d[1], d[2], c23);
    cross3(d[2], d[0], c31);
    cross3(d[0], d[1], c12);
    const double det = dot3(d[0], c23);
    for (int c = 0; c < 3; ++c) {
        g[1][c] = c23[c] / det;
        g[2][c] = c31[c] / det;
        g[3][c] = c12[c] / det;
        g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
    }
    *volume = std::fabs(det) / 6.0;
    return det;
}

// Unit-coefficient Whitney matrices in local orientation:
//   T[p][q] = int W_p . W_q with int l_a l_b = vol (1 + delta_ab) / 20,
//   S[p][q] = int curl W_p . curl W_q, curl W_ab = 2 grad l_a x grad l_b.
void whitney_matrices(const double g[4][3], double vol, double T[36], double S[36]) {
    double gg[4][4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) gg[a][b] = dot3(g[a], g[b]);
    auto m = [&](int a, int b) { return vol * (a == b ? 2.0 : 1.0) / 20.0; };
    double curl[6][3];
    for (int p = 0; p < 6; ++p) {
        cross3(g[kEdge[p][0]], g[kEdge[p][1]], curl[p]);
        for (int c = 0; c < 3; ++c) curl[p][c] *= 2.0;
    }
    for (int p = 0; p < 6; ++p) {
        const int a = kEdge[p][0], b = kEdge[p][1];
        for (int q = 0; q < 6; ++q) {
            const int c = kEdge[q][0], d = kEdge[q][1];
            T[6 * p + q] = m(a, c) * gg[b][d] - m(a, d) * gg[b][c] - m(b, c) * gg[a][d] + m(b, d) * gg[a][c];
            S[6 * p + q] = vol * dot3(curl[p], curl[q]);
        }
    }
}

struct Tri {
    int64_t a, b, c;
    bool operator<(const Tri& o) const {
        if (a != o.a) return a < o.a;
        if (b != o.b) return b < o.b;
        return c < o.c;
    }
    bool operator==(const Tri& o) const { return a == o.a && b == o.b && c == o.c; }
};

}  // namespace

int dd_build_host(dd_handle* h, const dd_mesh* mesh, const int32_t* part, int32_t n_sub) {
    const int64_t N = mesh->n_nodes, T = mesh->n_tets;
    h->n_nodes = N;
    h->n_tets = T;
    h->mu = mesh->mu;
    h->xyz.assign(mesh->xyz, mesh->xyz + 3 * N);
    h->tets.assign(mesh->tets, mesh->tets + 4 * T);
    h->eps.assign(T, 1.0);
    if (mesh->eps) h->eps.assign(mesh->eps, mesh->eps + T);
    h->part.assign(part, part + T);
    h->n_sub = n_sub;
    for (int64_t t = 0; t < 4 * T; ++t)
        if (h->tets[t] < 0 || h->tets[t] >= N) return h->fail(DD_ERR_ARG, "tet references a node out of range");
    for (int64_t t = 0; t < T; ++t)
        if (h->part[t] < 0 || h->part[t] >= n_sub) return h->fail(DD_ERR_ARG, "part[] out of range");
    for (int64_t t = 0; t < T; ++t)
        if (!(h->eps[t] > 0.0)) return h->fail(DD_ERR_ARG, "eps must be positive");
    if (!(h->mu > 0.0)) return h->fail(DD_ERR_ARG, "mu must be positive");

    // ---- edges: distinct (lo, hi) node pairs in lexicographic order ----------
    std::vector<int64_t> key(6 * T);
    for (int64_t t = 0; t < T; ++t)
        for (int k = 0; k < 6; ++k) {
            int64_t a = h->tets[4 * t + kEdge[k][0]], b = h->tets[4 * t + kEdge[k][1]];
            if (a == b) return h->fail(DD_ERR_MESH, "tet with a repeated node");
            key[6 * t + k] = std::min(a, b) * N + std::max(a, b);
        }
    std::vector<int64_t> ukey(key);
    std::sort(ukey.begin(), ukey.end());
    ukey.erase(std::unique(ukey.begin(), ukey.end()), ukey.end());
    h->n_edges = (int64_t)ukey.size();
    h->edges.resize(2 * h->n_edges);
    for (int64_t e = 0; e < h->n_edges; ++e) {
        h->edges[2 * e] = ukey[e] / N;
        h->edges[2 * e + 1] = ukey[e] % N;
    }
    auto edge_id = [&](int64_t a, int64_t b) {
        const int64_t k = std::min(a, b) * N + std::max(a, b);
        return (int64_t)(std::lower_bound(ukey.begin(), ukey.end(), k) - ukey.begin());
    };

    // ---- PEC: edges of triangles that belong to exactly one tet --------------
    std::vector<Tri> faces(4 * T);
    for (int64_t t = 0; t < T; ++t)
        for (int f = 0; f < 4; ++f) {
            int64_t v[3] = {h->tets[4 * t + kFace[f][0]], h->tets[4 * t + kFace[f][1]], h->tets[4 * t + kFace[f][2]]};
            std::sort(v, v + 3);
            faces[4 * t + f] = {v[0], v[1], v[2]};
        }
    std::sort(faces.begin(), faces.end());
    std::vector<uint8_t> pec(h->n_edges, 0);
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && faces[j] == faces[i]) ++j;
        if (j - i > 2) return h->fail(DD_ERR_MESH, "non-manifold face shared by more than two tets");
        if (j - i == 1) {
            pec[edge_id(faces[i].a, faces[i].b)] = 1;
            pec[edge_id(faces[i].a, faces[i].c)] = 1;
            pec[edge_id(faces[i].b, faces[i].c)] = 1;
        }
        i = j;
    }
    std::vector<int64_t> edge_dof(h->n_edges, -1);
    h->dof_edge.clear();
    for (int64_t e = 0; e < h->n_edges; ++e)
        if (!pec[e]) {
            edge_dof[e] = (int64_t)h->dof_edge.size();
            h->dof_edge.push_back(e);
        }
    h->n_dof = (int64_t)h->dof_edge.size();
    if (h->n_dof == 0) return h->fail(DD_ERR_MESH, "mesh has no interior edges");

    // ---- element matrices with global orientation lo -> hi --------------------
    h->tet_dof.resize(6 * T);
    h->That.resize(36 * T);
    h->Shat.resize(36 * T);
    h->grad.resize(12 * T);
    h->vol.resize(T);
    double bbox = 0.0;
    for (int64_t i = 0; i < 3 * N; ++i) bbox = std::max(bbox, std::fabs(h->xyz[i]));
    for (int64_t t = 0; t < T; ++t) {
        double X[12];
        for (int v = 0; v < 4; ++v)
            for (int c = 0; c < 3; ++c) X[3 * v + c] = h->xyz[3 * (int64_t)h->tets[4 * t + v] + c];
        double g[4][3], vol;
        const double det = tet_gradients(X, g, &vol);
        if (!(std::fabs(det) > 1e-13 * bbox * bbox * bbox) || !std::isfinite(det))
            return h->fail(DD_ERR_MESH, "degenerate tetrahedron " + std::to_string(t));
        h->vol[t] = vol;
        for (int v = 0; v < 4; ++v)
            for (int c = 0; c < 3; ++c) h->grad[12 * t + 3 * v + c] = g[v][c];
        double Tl[36], Sl[36];
        whitney_matrices(g, vol, Tl, Sl);
        int sgn[6];
        for (int k = 0; k < 6; ++k) {
            const int64_t a = h->tets[4 * t + kEdge[k][0]], b = h->tets[4 * t + kEdge[k][1]];
            sgn[k] = a < b ? 1 : -1;
            h->tet_dof[6 * t + k] = edge_dof[edge_id(a, b)];
        }
        for (int p = 0; p < 6; ++p)
            for (int q = 0; q < 6; ++q) {
                h->That[36 * t + 6 * p + q] = sgn[p] * sgn[q] * Tl[6 * p + q];
                h->Shat[36 * t + 6 * p + q] = sgn[p] * sgn[q] * Sl[6 * p + q];
            }
    }

    // ---- multiplicity: distinct subdomains touching each dof ------------------
    std::vector<int64_t> ds;  // dof * n_sub + sub
    ds.reserve(6 * T);
    for (int64_t t = 0; t < T; ++t)
        for (int k = 0; k < 6; ++k) {
            const int64_t d = h->tet_dof[6 * t + k];
            if (d >= 0) ds.push_back(d * n_sub + h->part[t]);
        }
    std::sort(ds.begin(), ds.end());
    ds.erase(std::unique(ds.begin(), ds.end()), ds.end());
    std::vector<int32_t> mult(h->n_dof, 0);
    h->owner.assign(h->n_dof, -1);
    for (int64_t v : ds) {
        const int64_t d = v / n_sub;
        if (mult[d] == 0) h->owner[d] = (int32_t)(v % n_sub);
        ++mult[d];
    }

    // ---- local numbering [interior | interface | corner], each by dof id ------
    std::vector<std::vector<int64_t>> grp(3 * (size_t)n_sub);
    for (int64_t v : ds) {
        const int64_t d = v / n_sub;
        const int s = (int)(v % n_sub);
        const int gi = mult[d] == 1 ? 0 : (mult[d] == 2 ? 1 : 2);
        grp[3 * s + gi].push_back(d);  // ds is sorted by dof, so each group is sorted
    }
    h->nI.assign(n_sub, 0);
    h->nG.assign(n_sub, 0);
    h->nC.assign(n_sub, 0);
    h->sub_ptr.assign(n_sub + 1, 0);
    h->local_dof.clear();
    for (int s = 0; s < n_sub; ++s) {
        h->nI[s] = (int32_t)grp[3 * s].size();
        h->nG[s] = (int32_t)grp[3 * s + 1].size();
        h->nC[s] = (int32_t)grp[3 * s + 2].size();
        if (h->nI[s] + h->nG[s] == 0)
            return h->fail(DD_ERR_PARTITION, "subdomain " + std::to_string(s) + " has no r unknowns");
        for (int gi = 0; gi < 3; ++gi)
            h->local_dof.insert(h->local_dof.end(), grp[3 * s + gi].begin(), grp[3 * s + gi].end());
        h->sub_ptr[s + 1] = (int64_t)h->local_dof.size();
    }
    const int64_t n_local = h->sub_ptr[n_sub];

    // slot metadata
    h->slot_mult.assign(n_local, 0);
    h->slot_corner.assign(n_local, -1);
    h->slot_dof.resize(n_local);
    h->slot_own.assign(n_local, 0);
    h->owner_slot.assign(h->n_dof, -1);
    h->slot_sub.assign(n_local, 0);
    std::vector<int32_t>& slot_sub = h->slot_sub;
    for (int s = 0; s < n_sub; ++s)
        for (int64_t i = h->sub_ptr[s]; i < h->sub_ptr[s + 1]; ++i) {
            slot_sub[i] = s;
            const int64_t d = h->local_dof[i];
            h->slot_dof[i] = (int32_t)d;
            if (h->owner[d] == s) {
                h->slot_own[i] = 1;
                h->owner_slot[d] = i;
            }
        }

    // copies of every dof (slots in subdomain order; the first is the owner)
    h->copy_ptr.assign(h->n_dof + 1, 0);
    for (int64_t i = 0; i < n_local; ++i) ++h->copy_ptr[h->local_dof[i] + 1];
    for (int64_t d = 0; d < h->n_dof; ++d) h->copy_ptr[d + 1] += h->copy_ptr[d];
    h->copy_slot.assign(n_local, -1);
    {
        std::vector<int64_t> fill(h->copy_ptr.begin(), h->copy_ptr.end() - 1);
        for (int64_t i = 0; i < n_local; ++i) h->copy_slot[fill[h->local_dof[i]]++] = i;
    }

    // multipliers (m = 2) and corners (m >= 3), in dof order
    std::vector<int64_t> mult_idx(h->n_dof, -1), corner_idx(h->n_dof, -1);
    h->mult_dof.clear();
    h->corner_dof.clear();
    for (int64_t d = 0; d < h->n_dof; ++d) {
        if (mult[d] == 2) {
            mult_idx[d] = (int64_t)h->mult_dof.size();
            h->mult_dof.push_back(d);
        } else if (mult[d] >= 3) {
            corner_idx[d] = (int64_t)h->corner_dof.size();
            h->corner_dof.push_back(d);
        }
    }
    const int64_t nl = (int64_t)h->mult_dof.size(), nc = (int64_t)h->corner_dof.size();
    h->mult_sub.assign(2 * nl, -1);
    h->mult_loc.assign(2 * nl, -1);
    h->mult_slot.assign(2 * nl, -1);
    std::vector<int64_t> ccount(nc + 1, 0);
    for (int64_t i = 0; i < n_local; ++i) {
        const int64_t d = h->local_dof[i];
        const int s = slot_sub[i];
        if (mult_idx[d] >= 0) {
            const int64_t m = mult_idx[d];
            const int side = (h->mult_sub[2 * m] < 0) ? 0 : 1;  // slots visited in subdomain order
            h->mult_sub[2 * m + side] = s;
            h->mult_loc[2 * m + side] = (int32_t)(i - h->sub_ptr[s]);
            h->mult_slot[2 * m + side] = i;
            h->slot_mult[i] = side == 0 ? (int32_t)(m + 1) : -(int32_t)(m + 1);
        } else if (corner_idx[d] >= 0) {
            h->slot_corner[i] = (int32_t)corner_idx[d];
            ++ccount[corner_idx[d] + 1];
        }
    }
    h->corner_ptr.assign(nc + 1, 0);
    for (int64_t c = 0; c < nc; ++c) h->corner_ptr[c + 1] = h->corner_ptr[c] + ccount[c + 1];
    h->corner_slot.assign(h->corner_ptr[nc], -1);
    {
        std::vector<int64_t> fill(h->corner_ptr.begin(), h->corner_ptr.end() - 1);
        for (int64_t i = 0; i < n_local; ++i)  // subdomain order
            if (h->slot_corner[i] >= 0) h->corner_slot[fill[h->slot_corner[i]]++] = i;
    }
    // coupled-operator output order: the two sides of every multiplier, then the corner copies
    h->slot_upos.assign(n_local, -1);
    for (int64_t k = 0; k < 2 * nl; ++k) h->slot_upos[h->mult_slot[k]] = (int32_t)k;
    for (int64_t k = 0; k < h->corner_ptr[nc]; ++k) h->slot_upos[h->corner_slot[k]] = (int32_t)(2 * nl + k);

    // ---- subassembled local CSR (rows = slots, per subdomain) -----------------
    std::vector<std::vector<int64_t>> tets_of(n_sub);
    for (int64_t t = 0; t < T; ++t) tets_of[h->part[t]].push_back(t);
    std::vector<int32_t> loc_of(h->n_dof, -1);
    h->row_ptr.assign(n_local + 1, 0);
    h->col_loc.clear();
    h->col_dof.clear();
    h->Tval.clear();
    h->Sval.clear();
    h->eps_contrib = 0;
    h->mats.resize(n_sub);
    h->max_nr = h->max_ns = 0;
    int64_t moff = 0;
    struct Trip {
        int64_t key;
        double t, s;
    };
    std::vector<Trip> trip;
    for (int s = 0; s < n_sub; ++s) {
        const int64_t base = h->sub_ptr[s];
        const int32_t ns = (int32_t)(h->sub_ptr[s + 1] - base);
        for (int32_t i = 0; i < ns; ++i) loc_of[h->local_dof[base + i]] = i;
        trip.clear();
        for (int64_t t : tets_of[s]) {
            for (int p = 0; p < 6; ++p) {
                const int64_t dp = h->tet_dof[6 * t + p];
                if (dp < 0) continue;
                for (int q = 0; q < 6; ++q) {
                    const int64_t dq = h->tet_dof[6 * t + q];
                    if (dq < 0) continue;
                    trip.push_back({(int64_t)loc_of[dp] * ns + loc_of[dq], h->eps[t] * h->That[36 * t + 6 * p + q],
                                    h->Shat[36 * t + 6 * p + q] / h->mu});
                }
            }
        }
        std::stable_sort(trip.begin(), trip.end(), [](const Trip& a, const Trip& b) { return a.key < b.key; });
        h->eps_contrib += (int64_t)trip.size();
        for (size_t i = 0; i < trip.size();) {
            size_t j = i;
            double tv = 0.0, sv = 0.0;
            while (j < trip.size() && trip[j].key == trip[i].key) {
                tv += trip[j].t;
                sv += trip[j].s;
                ++j;
            }
            const int64_t row = trip[i].key / ns, col = trip[i].key % ns;
            h->col_loc.push_back((int32_t)col);
            h->col_dof.push_back((int32_t)h->local_dof[base + col]);
            h->Tval.push_back(tv);
            h->Sval.push_back(sv);
            ++h->row_ptr[base + row + 1];
            i = j;
        }
        for (int32_t i = 0; i < ns; ++i) loc_of[h->local_dof[base + i]] = -1;
        MatDesc md;
        md.moff = moff;
        md.voff = base;
        md.nI = h->nI[s];
        md.nr = h->nI[s] + h->nG[s];
        md.ns = ns;
        md.ld = (ns + 3) / 4 * 4;
        if (s < h->n_sub_real) {
            moff += (int64_t)ns * md.ld;
        } else {   // ensemble copy: the same local matrix as member 0's subdomain
            const MatDesc& m0 = h->mats[s % h->n_sub_real];
            if (m0.ns != md.ns || m0.nI != md.nI || m0.nr != md.nr) throw std::runtime_error("ensemble copy differs");
            md.moff = m0.moff;
        }
        h->mats[s] = md;
        h->max_nr = std::max(h->max_nr, md.nr);
        h->max_ns = std::max(h->max_ns, md.ns);
    }
    for (int64_t i = 0; i < n_local; ++i) h->row_ptr[i + 1] += h->row_ptr[i];
    h->dense_elems = moff;
    // the dense K~cc^-1 serves the Schur CG only; an ensemble (coupled GMRES) has none
    h->ldc = h->members > 1 ? 0 : (int32_t)((nc + 3) / 4 * 4);

    // ---- interface tangential mass on the multiplier edges (MFETI-DP2) ---------
    // faces shared by tets of two subdomains; CSR over multipliers (block diagonal
    // by subdomain pair: the edges of such a face join exactly that pair)
    {
        struct FaceOwner {
            int64_t a, b, c;
            int32_t s;
            bool operator<(const FaceOwner& o) const {
                return a != o.a ? a < o.a : (b != o.b ? b < o.b : (c != o.c ? c < o.c : s < o.s));
            }
        };
        std::vector<FaceOwner> fo(4 * T);
        for (int64_t t = 0; t < T; ++t)
            for (int f = 0; f < 4; ++f) {
                int64_t v[3] = {h->tets[4 * t + kFace[f][0]], h->tets[4 * t + kFace[f][1]], h->tets[4 * t + kFace[f][2]]};
                std::sort(v, v + 3);
                fo[4 * t + f] = {v[0], v[1], v[2], h->part[t]};
            }
        std::sort(fo.begin(), fo.end());
        struct MT {
            int64_t k, l;
            double v;
        };
        std::vector<MT> mt;
        for (size_t i = 0; i + 1 < fo.size(); ++i) {
            const FaceOwner& x = fo[i];
            const FaceOwner& y = fo[i + 1];
            if (x.a != y.a || x.b != y.b || x.c != y.c || x.s == y.s) continue;
            const int64_t ev[3] = {edge_id(x.a, x.b), edge_id(x.b, x.c), edge_id(x.a, x.c)};
            int64_t mk[3];
            for (int e = 0; e < 3; ++e) {
                const int64_t d = edge_dof[ev[e]];
                mk[e] = d >= 0 ? mult_idx[d] : -1;
            }
            double M[9];
            face_mass(&h->xyz[3 * x.a], &h->xyz[3 * x.b], &h->xyz[3 * x.c], M);
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q)
                    if (mk[p] >= 0 && mk[q] >= 0) mt.push_back({mk[p], mk[q], M[3 * p + q]});
        }
        std::sort(mt.begin(), mt.end(), [](const MT& u, const MT& v) { return u.k != v.k ? u.k < v.k : u.l < v.l; });
        h->mt_ptr.assign(nl + 1, 0);
        h->mt_col.clear();
        h->mt_val.clear();
        for (size_t i = 0; i < mt.size();) {
            size_t j = i;
            double v = 0.0;
            while (j < mt.size() && mt[j].k == mt[i].k && mt[j].l == mt[i].l) v += mt[j++].v;
            h->mt_col.push_back((int32_t)mt[i].l);
            h->mt_val.push_back(v);
            ++h->mt_ptr[mt[i].k + 1];
            i = j;
        }
        for (int64_t k = 0; k < nl; ++k) h->mt_ptr[k + 1] += h->mt_ptr[k];
    }

    build_sym(h);
    build_tc(h);
    h->sym_ok = sym_smem_bytes(h) <= 227 * 1024;

    // ---- batched GEMV task lists (default tiles; dd_autotune may change them) ------
    for (int mode = 0; mode < GEMV_NMODES; ++mode) {
        std::vector<GemvTask> cap;
        build_tasks(h, mode, kMinRowsPerTask, cap);
        h->task_cap[mode] = cap.size();
        for (int p = 0; p < 2; ++p) {
            h->tile[p][mode] = TileCfg{p == 0 ? kLprF64[mode] : kLprF32[mode], kRowsPerMode[mode]};
            build_tasks(h, mode, kRowsPerMode[mode], h->tasks[p][mode]);
        }
    }
    return DD_OK;
}

// CTA tasks of a batched GEMV: the mode's row range of every subdomain (or of
// the coarse matrix) cut into chunks of `rows` rows.
void build_tasks(const dd_handle* h, int mode, int rows, std::vector<GemvTask>& tl) {
    tl.clear();
    if (mode == GEMV_COARSE) {
        if (h->ldc == 0) return;   // no dense K~cc^-1 (ensemble)
        const int64_t nc = (int64_t)h->corner_dof.size();
        for (int64_t r0 = 0; r0 < nc; r0 += rows)
            tl.push_back({0, (int32_t)r0, (int32_t)std::min<int64_t>(nc, r0 + rows), 0});
        return;
    }
    // ensemble: the copies of a subdomain one after the other (they read the same matrix)
    const int R = std::max(1, h->members), nsr = h->n_sub / R;
    for (int q = 0; q < h->n_sub; ++q) {
        const int s = (q % R) * nsr + q / R;
        const MatDesc& md = h->mats[s];
        int32_t r0 = 0, r1 = 0;
        if (mode == GEMV_LOCAL) { r0 = 0; r1 = md.ns; }
        if (mode == GEMV_SCHUR_C) { r0 = md.nr; r1 = md.ns; }
        if (mode == GEMV_CORNER) { r0 = md.nI; r1 = md.nr; }
        if (mode == GEMV_RECOVER) { r0 = 0; r1 = md.nr; }
        if (mode == GEMV_SCHUR_G) { r0 = md.nI; r1 = md.nr; }
        if (mode == GEMV_COUPLED) { r0 = md.nI; r1 = md.ns; }
        for (int32_t a = r0; a < r1; a += rows) tl.push_back({s, a, std::min(r1, a + rows), 0});
    }
}

int dd_locate_probes(dd_handle* h, int32_t n, const double* p) {
    h->probe_dof.assign(6 * (size_t)n, 0);
    h->probe_w.assign(18 * (size_t)n, 0.0);
    for (int32_t k = 0; k < n; ++k) {
        int64_t found = -1;
        double lam[4] = {0, 0, 0, 0};
        for (int64_t t = 0; t < h->n_tets && found < 0; ++t) {
            const double* g = &h->grad[12 * t];
            const double* x0 = &h->xyz[3 * (int64_t)h->tets[4 * t]];
            const double dx[3] = {p[3 * k] - x0[0], p[3 * k + 1] - x0[1], p[3 * k + 2] - x0[2]};
            double l[4];
            l[1] = dot3(g + 3, dx);
            l[2] = dot3(g + 6, dx);
            l[3] = dot3(g + 9, dx);
            l[0] = 1.0 - l[1] - l[2] - l[3];
            if (l[0] >= -1e-12 && l[1] >= -1e-12 && l[2] >= -1e-12 && l[3] >= -1e-12) {
                found = t;
                std::memcpy(lam, l, sizeof(l));
            }
        }
        if (found < 0) return h->fail(DD_ERR_ARG, "probe " + std::to_string(k) + " lies outside the mesh");
        const double* g = &h->grad[12 * found];
        for (int e = 0; e < 6; ++e) {
            const int a = kEdge[e][0], b = kEdge[e][1];
            const int64_t va = h->tets[4 * found + a], vb = h->tets[4 * found + b];
            const double sg = va < vb ? 1.0 : -1.0;
            const int64_t d = h->tet_dof[6 * found + e];
            h->probe_dof[6 * k + e] = d >= 0 ? (int32_t)d : 0;
            for (int c = 0; c < 3; ++c)
                h->probe_w[18 * k + 3 * e + c] = d >= 0 ? sg * (lam[a] * g[3 * b + c] - lam[b] * g[3 * a + c]) : 0.0;
        }
    }
    h->n_probe = n;
    return DD_OK;
}

// Particle set-up: faces (sorted node triples), the face opposite each local
// vertex of every tet, tet adjacency across faces, the discrete curl's edge
// list per face, and the boundary tet holding each injection point.
int dd_build_beam(dd_handle* h, const dd_beam* beam) {
    const int64_t T = h->n_tets, N = h->n_nodes, np = beam->n_particles;
    // faces
    std::vector<std::pair<Tri, int64_t>> fl(4 * T);
    for (int64_t t = 0; t < T; ++t)
        for (int f = 0; f < 4; ++f) {
            int64_t v[3] = {h->tets[4 * t + kFace[f][0]], h->tets[4 * t + kFace[f][1]], h->tets[4 * t + kFace[f][2]]};
            std::sort(v, v + 3);
            fl[4 * t + f] = {Tri{v[0], v[1], v[2]}, 4 * t + f};
        }
    std::sort(fl.begin(), fl.end(), [](const auto& a, const auto& b) {
        return a.first < b.first || (a.first == b.first && a.second < b.second);
    });
    h->tet_face.assign(4 * T, -1);
    h->tet_nbr.assign(4 * T, -1);
    h->face_nodes.clear();
    int64_t nf = 0;
    for (size_t i = 0; i < fl.size();) {
        size_t j = i + 1;
        while (j < fl.size() && fl[j].first == fl[i].first) ++j;
        h->face_nodes.push_back((int32_t)fl[i].first.a);
        h->face_nodes.push_back((int32_t)fl[i].first.b);
        h->face_nodes.push_back((int32_t)fl[i].first.c);
        for (size_t k = i; k < j; ++k) h->tet_face[fl[k].second] = (int32_t)nf;
        if (j - i == 2) {
            h->tet_nbr[fl[i].second] = (int32_t)(fl[i + 1].second / 4);
            h->tet_nbr[fl[i + 1].second] = (int32_t)(fl[i].second / 4);
        }
        ++nf;
        i = j;
    }
    h->n_faces = nf;
    // discrete curl: dofs of edges (a,b), (b,c), (a,c) of every sorted face
    std::vector<int64_t> key(h->n_edges);
    for (int64_t e = 0; e < h->n_edges; ++e) key[e] = h->edges[2 * e] * N + h->edges[2 * e + 1];
    std::vector<int64_t> edge_dof(h->n_edges, -1);
    for (int64_t d = 0; d < h->n_dof; ++d) edge_dof[h->dof_edge[d]] = d;
    auto dof_of = [&](int64_t a, int64_t b) {
        const int64_t e = std::lower_bound(key.begin(), key.end(), a * N + b) - key.begin();
        return (int32_t)edge_dof[e];
    };
    h->face_edge.resize(3 * nf);
    for (int64_t f = 0; f < nf; ++f) {
        const int64_t a = h->face_nodes[3 * f], b = h->face_nodes[3 * f + 1], c = h->face_nodes[3 * f + 2];
        h->face_edge[3 * f] = dof_of(a, b);
        h->face_edge[3 * f + 1] = dof_of(b, c);
        h->face_edge[3 * f + 2] = dof_of(a, c);
    }
    // injection tets: candidates are the tets with a wall face, binned on a coarse grid
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], h->xyz[3 * i + c]);
            hi[c] = std::max(hi[c], h->xyz[3 * i + c]);
        }
    const int G = 32;
    auto cell = [&](double x, int c) {
        const double w = (hi[c] - lo[c]) > 0 ? (hi[c] - lo[c]) : 1.0;
        return std::min(G - 1, std::max(0, (int)((x - lo[c]) / w * G)));
    };
    std::vector<std::vector<int32_t>> bins((size_t)G * G * G);
    for (int64_t t = 0; t < T; ++t) {
        bool wall = false;
        for (int f = 0; f < 4; ++f) wall |= h->tet_nbr[4 * t + f] < 0;
        if (!wall) continue;
        double tl[3] = {1e300, 1e300, 1e300}, th[3] = {-1e300, -1e300, -1e300};
        for (int v = 0; v < 4; ++v)
            for (int c = 0; c < 3; ++c) {
                const double x = h->xyz[3 * (int64_t)h->tets[4 * t + v] + c];
                tl[c] = std::min(tl[c], x);
                th[c] = std::max(th[c], x);
            }
        for (int i = cell(tl[0] - 1e-9, 0); i <= cell(th[0] + 1e-9, 0); ++i)
            for (int j = cell(tl[1] - 1e-9, 1); j <= cell(th[1] + 1e-9, 1); ++j)
                for (int k = cell(tl[2] - 1e-9, 2); k <= cell(th[2] + 1e-9, 2); ++k)
                    bins[((size_t)i * G + j) * G + k].push_back((int32_t)t);   // tets visited in id order
    }
    h->p_x.assign(beam->x_inj, beam->x_inj + 3 * np);
    h->p_v.assign(beam->v_inj, beam->v_inj + 3 * np);
    h->p_t.assign(beam->t_inj, beam->t_inj + np);
    h->p_tet.assign(np, -1);
    for (int64_t p = 0; p < np; ++p) {
        const double* x = &h->p_x[3 * p];
        if (!(h->p_t[p] >= 0.0)) return h->fail(DD_ERR_ARG, "negative injection time");
        const auto& cand = bins[((size_t)cell(x[0], 0) * G + cell(x[1], 1)) * G + cell(x[2], 2)];
        for (int32_t t : cand) {
            const double* g = &h->grad[12 * (int64_t)t];
            const double* x0 = &h->xyz[3 * (int64_t)h->tets[4 * (int64_t)t]];
            const double dx[3] = {x[0] - x0[0], x[1] - x0[1], x[2] - x0[2]};
            const double l1 = dot3(g + 3, dx), l2 = dot3(g + 6, dx), l3 = dot3(g + 9, dx);
            const double l0 = 1.0 - l1 - l2 - l3;
            if (l0 >= -1e-12 && l1 >= -1e-12 && l2 >= -1e-12 && l3 >= -1e-12) {
                h->p_tet[p] = t;
                break;
            }
        }
        if (h->p_tet[p] < 0)
            return h->fail(DD_ERR_ARG, "injection point " + std::to_string(p) + " is not on the mesh boundary");
    }
    h->n_particles = np;
    h->pq = beam->q;
    h->pqm = beam->qm;
    return DD_OK;
}

// Map of the local mass values onto the element matrices, for dd_set_eps:
// entry p of Tval (subdomain by subdomain, rows and columns in local order,
// as assembled above) receives the element-matrix entries idx[ptr[p]] ..
// idx[ptr[p+1]-1] (36 t + 6 a + b, scaled by eps[t]), listed in the order the
// host assembly adds them (tets ascending, then a, b), so that a device
// re-assembly reproduces the host's sums bitwise.
void build_eps_map(const dd_handle* h, std::vector<int64_t>& ptr, std::vector<int32_t>& idx) {
    const int n_sub = h->n_sub;
    std::vector<std::vector<int64_t>> tets_of(n_sub);
    for (int64_t t = 0; t < h->n_tets; ++t) tets_of[h->part[t]].push_back(t);
    std::vector<int32_t> loc_of(h->n_dof, -1);
    ptr.assign(1, 0);
    idx.clear();
    idx.reserve((size_t)h->eps_contrib);
    struct Ent {
        int64_t key;
        int32_t el;
    };
    std::vector<Ent> ent;
    for (int s = 0; s < n_sub; ++s) {
        const int64_t base = h->sub_ptr[s];
        const int32_t ns = (int32_t)(h->sub_ptr[s + 1] - base);
        for (int32_t i = 0; i < ns; ++i) loc_of[h->local_dof[base + i]] = i;
        ent.clear();
        for (int64_t t : tets_of[s])
            for (int a = 0; a < 6; ++a) {
                const int64_t da = h->tet_dof[6 * t + a];
                if (da < 0) continue;
                for (int b = 0; b < 6; ++b) {
                    const int64_t db = h->tet_dof[6 * t + b];
                    if (db < 0) continue;
                    ent.push_back({(int64_t)loc_of[da] * ns + loc_of[db], (int32_t)(36 * t + 6 * a + b)});
                }
            }
        std::stable_sort(ent.begin(), ent.end(), [](const Ent& x, const Ent& y) { return x.key < y.key; });
        for (size_t i = 0; i < ent.size();) {
            size_t j = i;
            while (j < ent.size() && ent[j].key == ent[i].key) idx.push_back(ent[j++].el);
            ptr.push_back((int64_t)idx.size());
            i = j;
        }
        for (int32_t i = 0; i < ns; ++i) loc_of[h->local_dof[base + i]] = -1;
    }
}
