// Marching cubes on a brick level (Sec. 4.6): the zero level set of u as a
// welded, consistently oriented triangle mesh.
//
// A cell is the cube of 8 voxel centres with lower corner voxel g (corner
// c = dx + 2 dy + 4 dz at g + (dx, dy, dz)); cells are owned by the brick of g
// and extracted for active bricks whose 8 corners all exist (active or frozen
// bricks).  Per cell:
//   * corner c is inside when u < 0;
//   * an edge (voxel p, axis a) crosses when its two ends differ; the crossing
//     lies at t = u_p / (u_p - u_q), coordinates o + ((g + 0.5) + t) h on a and
//     o + (g + 0.5) h on the other axes, FP32 with one rounding per operation;
//   * on each face, corners counter-clockwise seen from outside the cell, the
//     crossing where the boundary enters the inside region is joined to the next
//     one where it leaves; a face with four crossings takes the next exit when
//     ((u_a + u_b) + (u_c + u_d)) >= 0 over its corners in cell order (inside
//     corners apart), else the previous one (inside corners connected) -- the
//     neighbouring cell sees the same four values in the same order;
//   * the joins form closed loops, counter-clockwise seen from u >= 0; each loop
//     (started at its crossing on the lowest cell edge, index 4 a + the other two
//     base bits) is triangulated by the minimum-area dynamic programme
//       C[i][j] = min_{i<m<j} (C[i][m] + C[m][j]) + |(P_m - P_i) x (P_j - P_i)|
//     (FP32, ties to the smallest m) without chords between two crossings on a
//     common cell face; a loop that has no such triangulation is fanned around
//     its centroid (the cell's one extra vertex; later such loops in the same
//     cell fall back to the unconstrained programme).
// Vertex ids: 4 slot + a for the crossing on edge (slot, a), 4 slot + 3 for a
// cell's centroid; vertices are numbered by increasing id, triangles come in
// cell order.  Passes:
//   classify  one bit per cell whose corners change sign (a warp ballot per word);
//   compact   the crossing cells into a list in cell order (exclusive scan of the
//             words' popcounts; rank = word prefix + popcount of the lower bits),
//             then an order of the list grouped by the cells' corner signs (one
//             stable radix pass), in which the count pass takes the cells;
//   count     per listed cell: the loops and their triangulation; the triangles are
//             kept as edge-index triples in a per-cell record and the vertex ids
//             they reference are set in a bit set (4 ids per voxel slot);
//   scans     of the vertex bit set's word popcounts (vertex rank, as above) and of
//             the listed cells' triangle counts (triangle offsets);
//   write     per listed cell: triangles from its record, vertex positions.
// Only a few per cent of the cells cross the surface: listing them keeps the
// lanes of a warp busy in the loop triangulation, grouping them by sign pattern
// keeps those lanes on one path, and the record spares the write pass from
// repeating the triangulation.  Results go to list positions: cell order holds.
#include <math.h>

#include <unordered_map>
#include <vector>

#include "tgv_internal.cuh"
#include "tgv_zorder.cuh"

namespace {

constexpr int kMaxPoly = 12;

// counter-clockwise corner order of the faces -x, +x, -y, +y, -z, +z seen from outside
__constant__ int8_t c_face[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};

__device__ __forceinline__ int edge_of(int c0, int c1)
{
    const int lo = min(c0, c1), x = c0 ^ c1;
    const int a = x == 1 ? 0 : (x == 2 ? 1 : 2);
    // the two other corner bits of the lower corner, in axis order
    const int m = a == 0 ? (lo >> 1) : (a == 1 ? ((lo & 1) | ((lo >> 2) << 1)) : (lo & 3));
    return 4 * a + m;
}

__device__ __forceinline__ void edge_base(int e, int* base, int* axis)
{
    const int a = e >> 2, m = e & 3;
    *axis = a;
    *base = a == 0 ? 2 * (m & 1) + 4 * (m >> 1) : (a == 1 ? (m & 1) + 4 * (m >> 1) : m);
}

__device__ __forceinline__ bool on_common_face(int e1, int e2)
{
    int b1, a1, b2, a2;
    edge_base(e1, &b1, &a1);
    edge_base(e2, &b2, &a2);
    for (int f = 0; f < 3; ++f)
        if (f != a1 && f != a2 && ((b1 >> f) & 1) == ((b2 >> f) & 1)) return true;
    return false;
}

struct MeshArgs {
    const float* u;
    const int32_t* coords;  // 3 * (nb + nf)
    const int32_t* up7;     // nb x 7: bricks at +x, +y, +xy, +z, +xz, +yz, +xyz (-1 none)
    int64_t nb;
    float o[3], h;
    uint32_t* vbits;        // bit set over the vertex ids (4 per voxel slot)
    const uint32_t* vrank;  // exclusive prefix of the words' popcounts
    const uint32_t* cells;  // the crossing cells in cell order (ncross)
    const uint64_t* order;  // list positions grouped by corner signs: code << 32 | position
    int64_t ncross;
    uint32_t* tcount;       // per listed cell: triangle count, then exclusive offsets
    struct MeshRec* rec;    // per listed cell
    float* verts;
    int32_t* tris;
};

// The triangles of one listed cell: triangle t is the edge-index triple
// (e0 | e1 << 4 | e2 << 8) at bits 12 (t % 5) of tri[t / 5] (12 = the centroid).
// At most 12 triangles: a loop of k crossings gives k - 2, or k around the
// centroid (once per cell), and the loops share the 12 cell edges.
struct MeshRec {
    uint64_t tri[3];
    float centre[3];
    uint32_t head;  // bits 0-11 crossing edges, 12 centroid used, 16-19 triangle count
};

// Everything about one cell.
struct Cell {
    int64_t slot[8];
    float uc[8];
    int g[3];  // global voxel coordinates of corner 0
    int ncross;
    int cross;  // bit e set: cell edge e crosses
    int8_t next[12];
};

__device__ bool load_cell(const MeshArgs& A, int64_t b, int l, Cell& C)
{
    const int i = l & 7, j = (l >> 3) & 7, k = l >> 6;
    for (int c = 0; c < 8; ++c) {
        const int x = i + (c & 1), y = j + ((c >> 1) & 1), z = k + (c >> 2);
        const int code = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
        const int64_t nbk = code == 0 ? b : (int64_t)A.up7[b * 7 + code - 1];
        if (nbk < 0) return false;
        C.slot[c] = nbk * TGV_BVOX + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
        C.uc[c] = A.u[C.slot[c]];
    }
    for (int a = 0; a < 3; ++a) C.g[a] = 8 * A.coords[3 * b + a] + (a == 0 ? i : (a == 1 ? j : k));
    return true;
}

// crossings and the entry -> exit joins of every face
__device__ void cell_topology(Cell& C)
{
    int in = 0;
    for (int c = 0; c < 8; ++c) in |= (C.uc[c] < 0.0f) << c;
    C.cross = 0;
    C.ncross = 0;
    if (in == 0 || in == 0xff) return;
    for (int e = 0; e < 12; ++e) {
        int base, a;
        edge_base(e, &base, &a);
        if (((in >> base) ^ (in >> (base | (1 << a)))) & 1) {
            C.cross |= 1 << e;
            C.ncross++;
        }
    }
    for (int e = 0; e < 12; ++e) C.next[e] = -1;
    for (int f = 0; f < 6; ++f) {
        int typ[4], pe[4], n = 0;
        for (int m = 0; m < 4; ++m) {
            const int c0 = c_face[f][m], c1 = c_face[f][(m + 1) & 3];
            const int i0 = (in >> c0) & 1, i1 = (in >> c1) & 1;
            typ[m] = i0 == i1 ? 0 : (i0 ? 2 : 1);  // 1 entry (into inside), 2 exit
            pe[m] = edge_of(c0, c1);
            n += typ[m] != 0;
        }
        if (n == 0) continue;
        bool connected = false;
        if (n == 4) {
            // the face's corners in cell order: sort four small integers
            int s[4] = {c_face[f][0], c_face[f][1], c_face[f][2], c_face[f][3]};
            for (int x = 1; x < 4; ++x)
                for (int y = x; y > 0 && s[y] < s[y - 1]; --y) {
                    const int t = s[y];
                    s[y] = s[y - 1];
                    s[y - 1] = t;
                }
            const float sum = __fadd_rn(__fadd_rn(C.uc[s[0]], C.uc[s[1]]), __fadd_rn(C.uc[s[2]], C.uc[s[3]]));
            connected = sum < 0.0f;
        }
        for (int m = 0; m < 4; ++m) {
            if (typ[m] != 1) continue;
            int p = -1;
            for (int d = 1; d < 4 && p < 0; ++d) {
                const int q = connected ? (m + 4 - d) & 3 : (m + d) & 3;
                if (typ[q] == 2) p = q;
            }
            if (p >= 0) C.next[pe[m]] = (int8_t)pe[p];
        }
    }
}

__device__ __forceinline__ void crossing_point(const MeshArgs& A, const Cell& C, int e, float P[3])
{
    int base, a;
    edge_base(e, &base, &a);
    const float up = C.uc[base], uq = C.uc[base | (1 << a)];
    const float t = __fdiv_rn(up, __fsub_rn(up, uq));
    const int g[3] = {C.g[0] + (base & 1), C.g[1] + ((base >> 1) & 1), C.g[2] + (base >> 2)};
    for (int c = 0; c < 3; ++c) {
        float s = __fadd_rn(__int2float_rn(g[c]), 0.5f);
        if (c == a) s = __fadd_rn(s, t);
        P[c] = __fadd_rn(A.o[c], __fmul_rn(s, A.h));
    }
}

__device__ __forceinline__ float area2(const float (*P)[3], int i, int m, int j)
{
    float e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = __fsub_rn(P[m][c], P[i][c]);
        e2[c] = __fsub_rn(P[j][c], P[i][c]);
    }
    const float cx = __fsub_rn(__fmul_rn(e1[1], e2[2]), __fmul_rn(e1[2], e2[1]));
    const float cy = __fsub_rn(__fmul_rn(e1[2], e2[0]), __fmul_rn(e1[0], e2[2]));
    const float cz = __fsub_rn(__fmul_rn(e1[0], e2[1]), __fmul_rn(e1[1], e2[0]));
    return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz)));
}

// Minimum-area triangulation of loop P[0..k) (polygon-local triangles into tri).
// Returns k - 2, or -1 when every triangulation needs a chord along a cell face
// (only when constrained).
__device__ int triangulate(int k, const float (*P)[3], const int8_t* edges, bool constrained, int8_t (*tri)[3])
{
    if (k < 3) return k == 2 ? 0 : -1;  // two crossings: no triangle; one: no triangulation
    float Cst[kMaxPoly][kMaxPoly];
    int8_t best[kMaxPoly][kMaxPoly];
    // entries (i, j) with j > i only, each written before it is read
    for (int i = 0; i + 1 < k; ++i) {
        Cst[i][i + 1] = 0.0f;
        best[i][i + 1] = (int8_t)k;
    }
    for (int len = 2; len < k; ++len)
        for (int i = 0; i + len < k; ++i) {
            const int j = i + len;
            if (constrained && len < k - 1 && on_common_face(edges[i], edges[j])) {
                best[i][j] = -1;
                continue;
            }
            float bc = 0.0f;
            int bm = -1;
            for (int m = i + 1; m < j; ++m) {
                if (best[i][m] < 0 || best[m][j] < 0) continue;
                const float c = __fadd_rn(__fadd_rn(Cst[i][m], Cst[m][j]), area2(P, i, m, j));
                if (bm < 0 || c < bc) {
                    bc = c;
                    bm = m;
                }
            }
            Cst[i][j] = bc;
            best[i][j] = (int8_t)bm;
        }
    if (best[0][k - 1] < 0) return -1;
    // root first, then the (i, m) side, then the (m, j) side
    int8_t st[2 * kMaxPoly][2];
    int sp = 0, nt = 0;
    st[0][0] = 0;
    st[0][1] = (int8_t)(k - 1);
    sp = 1;
    while (sp > 0) {
        --sp;
        const int i = st[sp][0], j = st[sp][1];
        if (j - i < 2) continue;
        const int m = best[i][j];
        tri[nt][0] = (int8_t)i;
        tri[nt][1] = (int8_t)m;
        tri[nt][2] = (int8_t)j;
        ++nt;
        st[sp][0] = (int8_t)m;
        st[sp][1] = (int8_t)j;
        ++sp;
        st[sp][0] = (int8_t)i;
        st[sp][1] = (int8_t)m;
        ++sp;
    }
    return nt;
}

__device__ __forceinline__ uint64_t vid(const Cell& C, int e)
{
    if (e == 12) return 4 * (uint64_t)C.slot[0] + 3;
    int base, a;
    edge_base(e, &base, &a);
    return 4 * (uint64_t)C.slot[base] + (uint64_t)a;
}

// Triangulates every loop of the cell; emit(t0, t1, t2) gets cell edge indices
// (12 = the centroid).  Returns the triangle count; *centre receives the
// centroid when one was used (*used = true).
template <typename Emit>
__device__ int cell_triangles(const MeshArgs& A, const Cell& C, float centre[3], bool* used, Emit emit)
{
    *used = false;
    int done = 0, ntri = 0;
    for (int e0 = 0; e0 < 12; ++e0) {
        if (!((C.cross >> e0) & 1) || ((done >> e0) & 1)) continue;
        int8_t poly[kMaxPoly];
        int k = 0, e = e0;
        do {
            poly[k++] = (int8_t)e;
            done |= 1 << e;
            e = C.next[e];
        } while (e != e0 && e >= 0 && k < kMaxPoly);
        if (k == 3) {  // the programme's only triangulation, never constrained out
            emit(ntri++, poly[0], poly[1], poly[2]);
            continue;
        }
        float P[kMaxPoly][3];
        for (int v = 0; v < k; ++v) crossing_point(A, C, poly[v], P[v]);
        int8_t tri[kMaxPoly][3];
        int nt = triangulate(k, P, poly, true, tri);
        if (nt < 0 && !*used) {
            float c[3] = {0.0f, 0.0f, 0.0f};
            for (int v = 0; v < k; ++v)
                for (int q = 0; q < 3; ++q) c[q] = __fadd_rn(c[q], P[v][q]);
            for (int q = 0; q < 3; ++q) centre[q] = __fdiv_rn(c[q], (float)k);
            *used = true;
            for (int v = 0; v < k; ++v) emit(ntri++, poly[v], poly[(v + 1) % k], 12);
            continue;
        }
        if (nt < 0) nt = triangulate(k, P, poly, false, tri);
        for (int q = 0; q < nt; ++q) emit(ntri++, poly[tri[q][0]], poly[tri[q][1]], poly[tri[q][2]]);
    }
    return ntri;
}

// bit (cell & 31) of word[cell >> 5]: the cell exists and its corners change sign;
// code[cell]: its corner signs (bit c: corner c inside).  64 threads per brick, one per (i, j) column of 8 cells: the thread walks k = 0..7
// keeping the corner layer that the next cell shares; a warp holds four rows j, so
// each step k makes one word of the bit set by ballot.
__global__ void __launch_bounds__(256) mc_classify_kernel(const MeshArgs A, uint32_t* word, uint8_t* code)
{
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 6;
    if (b >= A.nb) return;  // whole warps: 64 threads per brick
    const int t = threadIdx.x & 63, i = t & 7, j = t >> 3;
    const int32_t* up = A.up7 + b * 7;
    const float* col[4];  // corner columns (dx, dy) = (c & 1, c >> 1): z = 0..7, then z = 8
    const float* top[4];
    bool lo_ok = true, hi_ok = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int x = i + (c & 1), y = j + (c >> 1);
        const int code = (x >> 3) | ((y >> 3) << 1);
        const int64_t nlo = code == 0 ? b : (int64_t)up[code - 1], nhi = up[code + 3];
        const int off = (x & 7) + 8 * (y & 7);
        lo_ok = lo_ok && nlo >= 0;
        hi_ok = hi_ok && nhi >= 0;
        col[c] = A.u + (nlo < 0 ? 0 : nlo) * TGV_BVOX + off;
        top[c] = A.u + (nhi < 0 ? 0 : nhi) * TGV_BVOX + off;
    }
    hi_ok = hi_ok && lo_ok;
    float v0[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v0[c] = lo_ok ? col[c][0] : 0.0f;
    uint32_t* w = word + b * (TGV_BVOX / 32) + (j >> 2);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool ok = k < 7 ? lo_ok : hi_ok;
        int in = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v1 = !ok ? 0.0f : (k < 7 ? col[c][64 * (k + 1)] : top[c][0]);
            in |= ((v0[c] < 0.0f) << c) | ((v1 < 0.0f) << (c + 4));
            v0[c] = v1;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, ok && in != 0 && in != 0xff);
        if ((threadIdx.x & 31) == 0) w[2 * k] = m;
        code[b * TGV_BVOX + t + 64 * k] = (uint8_t)in;
    }
}

// cnt[w] = popcount(word[w]) for w < nw, cnt[nw] = 0 (the exclusive scan of cnt then
// ranks the set bits)
__global__ void mc_popc_kernel(const uint32_t* word, int64_t nw, uint32_t* cnt)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) cnt[w] = (uint32_t)__popc(word[w]);
    else if (w == nw) cnt[w] = 0u;
}

__device__ __forceinline__ uint32_t bit_rank(const uint32_t* word, const uint32_t* prefix, uint64_t k)
{
    return prefix[k >> 5] + (uint32_t)__popc(word[k >> 5] & ((1u << (k & 31)) - 1u));
}

// cells[rank] = cell for every crossing cell, one thread per bit-set word, and the
// sort key (corner signs << 32 | rank) that groups the cells of one sign pattern
__global__ void mc_compact_kernel(const uint32_t* word, const uint32_t* prefix, int64_t nw, const uint8_t* code,
                                  uint32_t* cells, uint64_t* key)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    uint32_t m = word[w], r = prefix[w];
    while (m) {
        const uint32_t cell = (uint32_t)(32 * w) + (uint32_t)(__ffs(m) - 1);
        cells[r] = cell;
        key[r] = ((uint64_t)code[cell] << 32) | r;
        ++r;
        m &= m - 1;
    }
}

__device__ __forceinline__ void mark(uint32_t* bits, uint64_t id) { atomicOr(bits + (id >> 5), 1u << (id & 31)); }

// One thread per listed cell, cells of one sign pattern side by side (the same
// crossings and face joins: the lanes of a warp follow the same path); results
// are stored at the cell's list position, so the output keeps cell order.
__global__ void mc_count_kernel(const MeshArgs A)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.ncross) return;
    const int64_t i = (int64_t)(A.order[j] & 0xffffffffu);
    const uint32_t cell = A.cells[i];
    Cell C;
    uint32_t nt = 0, head = 0;
    uint64_t tri[3] = {0, 0, 0};
    float cen[3] = {0.0f, 0.0f, 0.0f};
    if (load_cell(A, cell / TGV_BVOX, (int)(cell % TGV_BVOX), C)) {
        cell_topology(C);
        if (C.ncross > 0) {
            bool used;
            nt = (uint32_t)cell_triangles(A, C, cen, &used, [&](int n, int e0, int e1, int e2) {
                if (n < 15) tri[n / 5] |= (uint64_t)(e0 | (e1 << 4) | (e2 << 8)) << (12 * (n % 5));
            });
            for (int e = 0; e < 12; ++e)
                if ((C.cross >> e) & 1) mark(A.vbits, vid(C, e));
            if (used) mark(A.vbits, vid(C, 12));
            head = (uint32_t)C.cross | ((uint32_t)used << 12) | (nt << 16);
        }
    }
    MeshRec& R = A.rec[i];
    for (int w = 0; w < 3; ++w) R.tri[w] = tri[w];
    for (int q = 0; q < 3; ++q) R.centre[q] = cen[q];
    R.head = head;
    A.tcount[i] = nt;
}

// Triangles of every listed cell at its offset, and the positions of the vertices
// it references: a crossing is written by each cell that has it (up to four), all
// with the same value (the same two corner values and voxel coordinates).
// (In list order: the pass does not triangulate, and its stores stay sequential.)
__global__ void mc_write_kernel(const MeshArgs A)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.ncross) return;
    const uint32_t o = A.tcount[i];
    const MeshRec& R = A.rec[i];
    const uint32_t head = R.head;
    const int nt = (int)(head >> 16);
    if (nt == 0) return;
    const uint32_t cell = A.cells[i];
    Cell C;
    if (!load_cell(A, cell / TGV_BVOX, (int)(cell % TGV_BVOX), C)) return;
    C.cross = (int)(head & 0xfffu);
    int32_t* T = A.tris + 3 * (int64_t)o;
    const uint32_t* B = A.vbits;
    for (int n = 0; n < nt; ++n) {
        const uint32_t code = (uint32_t)(R.tri[n / 5] >> (12 * (n % 5))) & 0xfffu;
        for (int q = 0; q < 3; ++q) T[3 * n + q] = (int32_t)bit_rank(B, A.vrank, vid(C, (code >> (4 * q)) & 15u));
    }
    if ((head >> 12) & 1u) {
        float* P = A.verts + 3 * (int64_t)bit_rank(B, A.vrank, vid(C, 12));
        for (int q = 0; q < 3; ++q) P[q] = R.centre[q];
    }
    for (int e = 0; e < 12; ++e) {
        if (!((C.cross >> e) & 1)) continue;
        float P[3];
        crossing_point(A, C, e, P);
        float* V = A.verts + 3 * (int64_t)bit_rank(B, A.vrank, vid(C, e));
        for (int q = 0; q < 3; ++q) V[q] = P[q];
    }
}

// ---- exclusive scan of uint32 (in place), three phases; returns the total on the host
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* warp_tot, uint32_t* total)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = w > 0 ? warp_tot[w - 1] : 0u;
    if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const uint32_t* in, int64_t n, uint32_t* tile_sums)
{
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    __shared__ uint32_t tot;
    block_exclusive(s, wt, threadIdx.x == 0 ? &tot : nullptr);
    __syncthreads();
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint32_t* sums, int64_t n, uint32_t* total)
{
    __shared__ uint32_t wt[32];
    __shared__ uint32_t carry, chunk_tot;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c = 0; c < n; c += kScanThreads) {
        const int64_t i = c + threadIdx.x;
        const uint32_t v = i < n ? sums[i] : 0u;
        const uint32_t ex = block_exclusive(v, wt, threadIdx.x == 0 ? &chunk_tot : nullptr);
        __syncthreads();
        if (i < n) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += chunk_tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(uint32_t* data, int64_t n, const uint32_t* tile_off)
{
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? data[base + k] : 0u;
        s += v[k];
    }
    uint32_t run = block_exclusive(s, wt, nullptr) + tile_off[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) {
            data[base + k] = run;
            run += v[k];
        }
}

}  // namespace

// exclusive scan of n uint32 in place; *total receives the sum (synchronises the stream)
tgv_status tgv_exclusive_scan_u32(tgv_domain* d, uint32_t* data, int64_t n, TgvScratch& tmp, uint64_t* total)
{
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    tgv_status st = tgv_scratch(d, tmp, sizeof(uint32_t) * (size_t)(tiles + 1));
    if (st != TGV_OK) return st;
    uint32_t* sums = (uint32_t*)tmp.ptr;
    if (tiles > 0) {
        scan_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, d->stream>>>(data, n, sums);
        scan_sums_kernel<<<1, kScanThreads, 0, d->stream>>>(sums, tiles, sums + tiles);
        scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, d->stream>>>(data, n, sums);
        d->launches += 3;
    } else {
        cudaMemsetAsync(sums, 0, sizeof(uint32_t), d->stream);
    }
    uint32_t t = 0;
    cudaError_t e = cudaMemcpyAsync(&t, sums + tiles, sizeof(uint32_t), cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if ((st = tgv_cuda_check(d, e, "exclusive scan")) != TGV_OK) return st;
    *total = t;
    return TGV_OK;
}

// Upper-neighbour rows (+x, +y, +xy, +z, +xz, +yz, +xyz) of the active bricks,
// from the level's brick coordinates; built once per level.
static tgv_status build_up7(tgv_domain* d, TgvLevel& L)
{
    if (L.up7) return TGV_OK;
    const int64_t na = L.nb + L.nf;
    std::unordered_map<uint64_t, int32_t> index;
    index.reserve((size_t)na * 2);
    auto key = [](int64_t x, int64_t y, int64_t z) -> uint64_t {
        const int64_t B = (int64_t)1 << 20;
        return ((uint64_t)(z + B) * (uint64_t)(2 * B) + (uint64_t)(y + B)) * (uint64_t)(2 * B) + (uint64_t)(x + B);
    };
    for (int64_t i = 0; i < na; ++i) index.emplace(key(L.coords[3 * i], L.coords[3 * i + 1], L.coords[3 * i + 2]), (int32_t)i);
    std::vector<int32_t> up((size_t)std::max<int64_t>(L.nb, 1) * 7, -1);
    for (int64_t b = 0; b < L.nb; ++b)
        for (int code = 1; code < 8; ++code) {
            auto it = index.find(key(L.coords[3 * b] + (code & 1), L.coords[3 * b + 1] + ((code >> 1) & 1),
                                     L.coords[3 * b + 2] + (code >> 2)));
            up[(size_t)b * 7 + code - 1] = it == index.end() ? -1 : it->second;
        }
    cudaError_t e = cudaMalloc(&L.up7, up.size() * 4);
    if (e != cudaSuccess) {
        cudaGetLastError();
        L.up7 = nullptr;
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "mesh neighbour table allocation failed");
    }
    d->bytes += (int64_t)up.size() * 4;
    e = cudaMemcpyAsync(L.up7, up.data(), up.size() * 4, cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "mesh neighbour table upload");
}

tgv_status tgv_mesh_extract(tgv_domain* d, TgvLevel& L, int64_t* nverts, int64_t* ntris)
{
    *nverts = *ntris = 0;
    tgv_status st = build_up7(d, L);
    if (st != TGV_OK) return st;
    const int64_t ncell = L.nb * TGV_BVOX, nids = 4 * (L.nb + L.nf) * TGV_BVOX;
    if (ncell == 0) {
        d->mesh_nv = d->mesh_nt = 0;
        return TGV_OK;
    }
    if (nids >= ((int64_t)1 << 32) - 1 || ncell >= ((int64_t)1 << 32) - 1)
        return tgv_fail(d, TGV_ERR_UNSUPPORTED, "level too large for 32-bit mesh indices");
    const int64_t nwv = (nids + 31) / 32, nwc = (ncell + 31) / 32;  // bit-set words
    if ((st = tgv_scratch(d, d->mesh_flags, sizeof(uint32_t) * (size_t)(2 * nwv + 1))) != TGV_OK) return st;
    if ((st = tgv_scratch(d, d->mesh_count, sizeof(uint32_t) * (size_t)(2 * nwc + 1) + (size_t)ncell)) != TGV_OK)
        return st;
    MeshArgs A;
    A.u = L.u;
    A.coords = L.coords_dev;
    A.up7 = L.up7;
    A.nb = L.nb;
    for (int a = 0; a < 3; ++a) A.o[a] = (float)L.origin[a];
    A.h = (float)L.h;
    A.vbits = (uint32_t*)d->mesh_flags.ptr;
    uint32_t* vcnt = A.vbits + nwv;
    A.vrank = vcnt;
    uint32_t* cword = (uint32_t*)d->mesh_count.ptr;
    uint32_t* ccnt = cword + nwc;
    uint8_t* code = (uint8_t*)(ccnt + nwc + 1);
    cudaError_t e = cudaMemsetAsync(A.vbits, 0, sizeof(uint32_t) * (size_t)nwv, d->stream);
    if ((st = tgv_cuda_check(d, e, "mesh scratch clear")) != TGV_OK) return st;
    mc_classify_kernel<<<(unsigned)((L.nb + 3) / 4), 256, 0, d->stream>>>(A, cword, code);
    mc_popc_kernel<<<(unsigned)((nwc + 256) / 256), 256, 0, d->stream>>>(cword, nwc, ccnt);
    d->launches += 2;
    if ((st = tgv_cuda_check(d, cudaGetLastError(), "mc_classify_kernel launch")) != TGV_OK) return st;
    uint64_t nc = 0, nv = 0, nt = 0;
    if ((st = tgv_exclusive_scan_u32(d, ccnt, nwc + 1, d->mesh_scan, &nc)) != TGV_OK) return st;
    // listed cells: cell ids, triangle counts (nc + 1), records, sort keys and the
    // sort's temporaries (16-byte aligned parts)
    const size_t ncz = (size_t)std::max<uint64_t>(nc, 1);
    auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t rec_off = up16(sizeof(uint32_t) * (2 * (size_t)nc + 1));
    const size_t key_off = up16(rec_off + sizeof(MeshRec) * ncz);
    const size_t tmp_off = key_off + 8 * ncz, hist_off = tmp_off + 8 * ncz;
    if ((st = tgv_scratch(d, d->mesh_cells, hist_off + 4 * (size_t)tgv_radix_hist_words((int64_t)ncz))) != TGV_OK)
        return st;
    char* base = (char*)d->mesh_cells.ptr;
    uint32_t* cells = (uint32_t*)base;
    uint64_t* keys = (uint64_t*)(base + key_off);
    A.cells = cells;
    A.order = keys;
    A.ncross = (int64_t)nc;
    A.tcount = cells + nc;
    A.rec = (MeshRec*)(base + rec_off);
    const unsigned lgrid = (unsigned)((nc + 127) / 128);
    if (nc > 0) {
        mc_compact_kernel<<<(unsigned)((nwc + 255) / 256), 256, 0, d->stream>>>(cword, ccnt, nwc, code, cells, keys);
        d->launches++;
        // group the cells by corner signs (one stable 8-bit pass: ties keep list order); the
        // count and write passes read the sorted keys where the pass left them
        uint64_t* sorted = keys;
        e = tgv_radix_sort_u64(keys, (uint64_t*)(base + tmp_off), (uint32_t*)(base + hist_off), (int64_t)nc, 32, 8,
                               d->stream, &d->launches, &sorted);
        if ((st = tgv_cuda_check(d, e, "mesh cell grouping")) != TGV_OK) return st;
        A.order = sorted;
        mc_count_kernel<<<lgrid, 128, 0, d->stream>>>(A);
        d->launches++;
    }
    mc_popc_kernel<<<(unsigned)((nwv + 256) / 256), 256, 0, d->stream>>>(A.vbits, nwv, vcnt);
    d->launches++;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(A.tcount + nc, 0, sizeof(uint32_t), d->stream);
    if ((st = tgv_cuda_check(d, e, "mc_count_kernel launch")) != TGV_OK) return st;
    if ((st = tgv_exclusive_scan_u32(d, vcnt, nwv + 1, d->mesh_scan, &nv)) != TGV_OK) return st;
    if ((st = tgv_exclusive_scan_u32(d, A.tcount, (int64_t)nc + 1, d->mesh_scan, &nt)) != TGV_OK) return st;
    if (nv >= ((uint64_t)1 << 31) || nt >= ((uint64_t)1 << 31))
        return tgv_fail(d, TGV_ERR_UNSUPPORTED, "mesh too large for 32-bit vertex indices");
    if ((st = tgv_scratch(d, d->mesh_v, sizeof(float) * 3 * (size_t)std::max<uint64_t>(nv, 1))) != TGV_OK) return st;
    if ((st = tgv_scratch(d, d->mesh_t, sizeof(int32_t) * 3 * (size_t)std::max<uint64_t>(nt, 1))) != TGV_OK) return st;
    A.verts = (float*)d->mesh_v.ptr;
    A.tris = (int32_t*)d->mesh_t.ptr;
    if (nc > 0) {
        mc_write_kernel<<<lgrid, 128, 0, d->stream>>>(A);
        d->launches++;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if ((st = tgv_cuda_check(d, e, "mc_write_kernel")) != TGV_OK) return st;
    d->mesh_nv = (int64_t)nv;
    d->mesh_nt = (int64_t)nt;
    *nverts = (int64_t)nv;
    *ntris = (int64_t)nt;
    return TGV_OK;
}
