// dg_refine.cu -- uniform (red) refinement of a triangulation, the paper's
// uniformrefine (Sec. 2.1): every triangle is cut into four by its edge
// midpoints and every boundary edge into two, so a split-square mesh stays a
// split-square mesh with the same diagonal.  Host code only (a one-off,
// O(ne) pass over a hash map of edges); the refined arrays then go through
// dg_mesh_upload like any other mesh.
#include <stdint.h>
#include <string.h>

#include <unordered_map>
#include <vector>

#include "dg_internal.cuh"

namespace {

inline uint64_t edge_key(int a, int b) {
    const uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
    return ((uint64_t)hi << 32) | lo;
}

// midpoint node of every edge, numbered from nv in the order the edges are
// first met (elements in order, local edges (0,1), (1,2), (2,0))
struct Midpoints {
    std::unordered_map<uint64_t, int> id;
    std::vector<int> ends;   // 2 per new node
    int nv;
    explicit Midpoints(int nv0, int ne) : nv(nv0) { id.reserve((size_t)ne * 2); }
    int get(int a, int b) {
        auto it = id.emplace(edge_key(a, b), nv + (int)(ends.size() / 2));
        if (it.second) {
            ends.push_back(a);
            ends.push_back(b);
        }
        return it.first->second;
    }
    int find(int a, int b) const {
        auto it = id.find(edge_key(a, b));
        return it == id.end() ? -1 : it->second;
    }
};

}  // namespace

extern "C" dg_status dg_mesh_refine(const double* nodes, int nv, const int* elems, int ne, const int* dirichlet,
                                    int nd, const int* neumann, int nn, double* nodes_out, int* nv_out,
                                    int* elems_out, int* ne_out, int* dirichlet_out, int* nd_out, int* neumann_out,
                                    int* nn_out) {
    if (!nodes || !elems || nv < 3 || ne < 1 || nd < 0 || nn < 0 || (nd > 0 && !dirichlet) ||
        (nn > 0 && !neumann) || !nv_out || !ne_out || !nd_out || !nn_out || ne > (1 << 27))
        return DG_ERR_INVALID_ARG;
    for (long t = 0; t < 3L * ne; ++t)
        if (elems[t] < 0 || elems[t] >= nv) return DG_ERR_MESH;
    Midpoints mid(nv, ne);
    std::vector<int> m(3 * (size_t)ne);
    for (int K = 0; K < ne; ++K)
        for (int f = 0; f < 3; ++f) m[3 * (size_t)K + f] = mid.get(elems[3 * K + f], elems[3 * K + (f + 1) % 3]);
    const long nnew = (long)mid.ends.size() / 2;
    if ((long)nv + nnew > (1L << 30)) return DG_ERR_INVALID_ARG;
    // boundary edges must be element edges
    for (int b = 0; b < nd + nn; ++b) {
        const int* e = b < nd ? dirichlet + 2 * b : neumann + 2 * (b - nd);
        if (e[0] < 0 || e[0] >= nv || e[1] < 0 || e[1] >= nv || mid.find(e[0], e[1]) < 0) return DG_ERR_MESH;
    }
    *nv_out = nv + (int)nnew;
    *ne_out = 4 * ne;
    *nd_out = 2 * nd;
    *nn_out = 2 * nn;
    if (!nodes_out) return DG_OK;   // sizes only
    if (!elems_out || (nd > 0 && !dirichlet_out) || (nn > 0 && !neumann_out)) return DG_ERR_INVALID_ARG;
    memcpy(nodes_out, nodes, sizeof(double) * 2 * (size_t)nv);
    for (long i = 0; i < nnew; ++i) {
        const int a = mid.ends[2 * i], b = mid.ends[2 * i + 1];
        nodes_out[2 * (nv + i)] = 0.5 * (nodes[2 * a] + nodes[2 * b]);
        nodes_out[2 * (nv + i) + 1] = 0.5 * (nodes[2 * a + 1] + nodes[2 * b + 1]);
    }
    for (int K = 0; K < ne; ++K) {
        const int a = elems[3 * K], b = elems[3 * K + 1], c = elems[3 * K + 2];
        const int mab = m[3 * (size_t)K], mbc = m[3 * (size_t)K + 1], mca = m[3 * (size_t)K + 2];
        const int child[4][3] = {{a, mab, mca}, {mab, b, mbc}, {mca, mbc, c}, {mab, mbc, mca}};
        for (int t = 0; t < 4; ++t)
            for (int v = 0; v < 3; ++v) elems_out[12 * (size_t)K + 3 * t + v] = child[t][v];
    }
    for (int b = 0; b < nd + nn; ++b) {
        const bool isd = b < nd;
        const int* e = isd ? dirichlet + 2 * b : neumann + 2 * (b - nd);
        int* o = isd ? dirichlet_out + 4 * b : neumann_out + 4 * (b - nd);
        const int mm = mid.find(e[0], e[1]);
        o[0] = e[0];
        o[1] = mm;
        o[2] = mm;
        o[3] = e[1];
    }
    return DG_OK;
}
