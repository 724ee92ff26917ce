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
// cell order.  Passes: count (per-cell triangle counts, referenced ids marked),
// two exclusive scans (vertex ranks, triangle offsets), write (triangles and the
// positions of the vertices each cell references).
#include <math.h>

#include <unordered_map>
#include <vector>

#include "tgv_internal.cuh"

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
    uint32_t* flags;        // 4 ids per voxel slot: marked, then exclusive ranks
    uint32_t* tcount;       // per cell: triangle count, then exclusive offsets
    float* verts;
    int32_t* tris;
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
    float Cst[kMaxPoly][kMaxPoly];
    int8_t best[kMaxPoly][kMaxPoly];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            Cst[i][j] = 0.0f;
            best[i][j] = j == i + 1 ? (int8_t)k : (int8_t)-1;
        }
    for (int len = 2; len < k; ++len)
        for (int i = 0; i + len < k; ++i) {
            const int j = i + len;
            if (constrained && len < k - 1 && on_common_face(edges[i], edges[j])) continue;
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

__global__ void mc_count_kernel(const MeshArgs A)
{
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= A.nb * TGV_BVOX) return;
    Cell C;
    uint32_t nt = 0;
    if (load_cell(A, cell / TGV_BVOX, (int)(cell % TGV_BVOX), C)) {
        cell_topology(C);
        if (C.ncross > 0) {
            float cen[3];
            bool used;
            nt = (uint32_t)cell_triangles(A, C, cen, &used, [](int, int, int, int) {});
            for (int e = 0; e < 12; ++e)
                if ((C.cross >> e) & 1) A.flags[vid(C, e)] = 1u;
            if (used) A.flags[vid(C, 12)] = 1u;
        }
    }
    A.tcount[cell] = nt;
}

// Triangles of every cell at its offset, and the positions of the vertices it
// references: a crossing is written by each cell that has it (up to four), all
// with the same value (the same two corner values and voxel coordinates).
__global__ void mc_write_kernel(const MeshArgs A)
{
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= A.nb * TGV_BVOX) return;
    const uint32_t o = A.tcount[cell], o1 = A.tcount[cell + 1];
    if (o1 == o) return;
    Cell C;
    if (!load_cell(A, cell / TGV_BVOX, (int)(cell % TGV_BVOX), C)) return;
    cell_topology(C);
    float cen[3];
    bool used;
    int32_t* T = A.tris + 3 * (int64_t)o;
    const uint32_t* F = A.flags;
    cell_triangles(A, C, cen, &used, [&](int n, int e0, int e1, int e2) {
        T[3 * n + 0] = (int32_t)F[vid(C, e0)];
        T[3 * n + 1] = (int32_t)F[vid(C, e1)];
        T[3 * n + 2] = (int32_t)F[vid(C, e2)];
    });
    if (used) {
        float* P = A.verts + 3 * (int64_t)F[vid(C, 12)];
        for (int q = 0; q < 3; ++q) P[q] = cen[q];
    }
    for (int e = 0; e < 12; ++e) {
        if (!((C.cross >> e) & 1)) continue;
        float P[3];
        crossing_point(A, C, e, P);
        float* V = A.verts + 3 * (int64_t)F[vid(C, e)];
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
    if ((st = tgv_scratch(d, d->mesh_flags, sizeof(uint32_t) * (size_t)nids)) != TGV_OK) return st;
    if ((st = tgv_scratch(d, d->mesh_count, sizeof(uint32_t) * (size_t)(ncell + 1))) != TGV_OK) return st;
    MeshArgs A;
    A.u = L.u;
    A.coords = L.coords_dev;
    A.up7 = L.up7;
    A.nb = L.nb;
    for (int a = 0; a < 3; ++a) A.o[a] = (float)L.origin[a];
    A.h = (float)L.h;
    A.flags = (uint32_t*)d->mesh_flags.ptr;
    A.tcount = (uint32_t*)d->mesh_count.ptr;
    cudaError_t e = cudaMemsetAsync(A.flags, 0, sizeof(uint32_t) * (size_t)nids, d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.tcount + ncell, 0, sizeof(uint32_t), d->stream);
    if ((st = tgv_cuda_check(d, e, "mesh scratch clear")) != TGV_OK) return st;
    const unsigned cgrid = (unsigned)((ncell + 127) / 128);
    mc_count_kernel<<<cgrid, 128, 0, d->stream>>>(A);
    d->launches++;
    if ((st = tgv_cuda_check(d, cudaGetLastError(), "mc_count_kernel launch")) != TGV_OK) return st;
    uint64_t nv = 0, nt = 0;
    if ((st = tgv_exclusive_scan_u32(d, A.flags, nids, d->mesh_scan, &nv)) != TGV_OK) return st;
    if ((st = tgv_exclusive_scan_u32(d, A.tcount, ncell + 1, d->mesh_scan, &nt)) != TGV_OK) return st;
    if (nv >= ((uint64_t)1 << 31) || nt >= ((uint64_t)1 << 31))
        return tgv_fail(d, TGV_ERR_UNSUPPORTED, "mesh too large for 32-bit vertex indices");
    if ((st = tgv_scratch(d, d->mesh_v, sizeof(float) * 3 * (size_t)std::max<uint64_t>(nv, 1))) != TGV_OK) return st;
    if ((st = tgv_scratch(d, d->mesh_t, sizeof(int32_t) * 3 * (size_t)std::max<uint64_t>(nt, 1))) != TGV_OK) return st;
    A.verts = (float*)d->mesh_v.ptr;
    A.tris = (int32_t*)d->mesh_t.ptr;
    mc_write_kernel<<<cgrid, 128, 0, d->stream>>>(A);
    d->launches++;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if ((st = tgv_cuda_check(d, e, "mc_write_kernel")) != TGV_OK) return st;
    d->mesh_nv = (int64_t)nv;
    d->mesh_nt = (int64_t)nt;
    *nverts = (int64_t)nv;
    *ntris = (int64_t)nt;
    return TGV_OK;
}
