// Structured hexahedral block as a face-addressed mesh (the convenience builder of the C ABI).
//
// Cells (i, j, k) are numbered i + nx (j + ny k), points (i, j, k) i + (nx+1)(j + (ny+1) k).
// Internal faces come first, ordered by (owner, neighbour), each quad's point loop turning
// right-handed about the normal from owner (lower index) to neighbour; then six boundary
// patches, each quad's normal pointing out of its cell:
//   side 0 x-min, 1 x-max (cells (j, k), j fastest), 2 y-min, 3 y-max ((i, k), i fastest),
//   4 z-min, 5 z-max ((i, j), i fastest).
// dim = 2 needs nz = 1 and makes the z sides EMPTY (plane strain).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "jfnk_gb300.h"

namespace {

struct HexFaces {
    std::vector<int32_t> ptr, pts, own, nei;
};

int64_t n_internal_faces(int64_t nx, int64_t ny, int64_t nz)
{
    return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
}

void build(int nx, int ny, int nz, HexFaces& h)
{
    const int px = nx + 1, py = ny + 1;
    auto pid = [&](int i, int j, int k) { return (int32_t)(i + px * (j + py * k)); };
    auto cid = [&](int i, int j, int k) { return (int32_t)(i + nx * (j + ny * k)); };
    struct F { int32_t o, n, q[4]; };
    std::vector<F> in;
    in.reserve((size_t)n_internal_faces(nx, ny, nz));
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                if (i + 1 < nx)
                    in.push_back({cid(i, j, k), cid(i + 1, j, k),
                                  {pid(i + 1, j, k), pid(i + 1, j + 1, k), pid(i + 1, j + 1, k + 1), pid(i + 1, j, k + 1)}});
                if (j + 1 < ny)
                    in.push_back({cid(i, j, k), cid(i, j + 1, k),
                                  {pid(i, j + 1, k), pid(i, j + 1, k + 1), pid(i + 1, j + 1, k + 1), pid(i + 1, j + 1, k)}});
                if (k + 1 < nz)
                    in.push_back({cid(i, j, k), cid(i, j, k + 1),
                                  {pid(i, j, k + 1), pid(i + 1, j, k + 1), pid(i + 1, j + 1, k + 1), pid(i, j + 1, k + 1)}});
            }
    std::stable_sort(in.begin(), in.end(), [](const F& a, const F& b) { return a.o != b.o ? a.o < b.o : a.n < b.n; });
    h.ptr.assign(1, 0);
    h.pts.clear();
    h.own.clear();
    h.nei.clear();
    auto push = [&](int32_t o, const int32_t* q) {
        for (int t = 0; t < 4; t++) h.pts.push_back(q[t]);
        h.ptr.push_back((int32_t)h.pts.size());
        h.own.push_back(o);
    };
    for (const F& f : in) {
        push(f.o, f.q);
        h.nei.push_back(f.n);
    }
    for (int k = 0; k < nz; k++)  // x-min
        for (int j = 0; j < ny; j++) {
            const int32_t q[4] = {pid(0, j, k), pid(0, j, k + 1), pid(0, j + 1, k + 1), pid(0, j + 1, k)};
            push(cid(0, j, k), q);
        }
    for (int k = 0; k < nz; k++)  // x-max
        for (int j = 0; j < ny; j++) {
            const int32_t q[4] = {pid(nx, j, k), pid(nx, j + 1, k), pid(nx, j + 1, k + 1), pid(nx, j, k + 1)};
            push(cid(nx - 1, j, k), q);
        }
    for (int k = 0; k < nz; k++)  // y-min
        for (int i = 0; i < nx; i++) {
            const int32_t q[4] = {pid(i, 0, k), pid(i + 1, 0, k), pid(i + 1, 0, k + 1), pid(i, 0, k + 1)};
            push(cid(i, 0, k), q);
        }
    for (int k = 0; k < nz; k++)  // y-max
        for (int i = 0; i < nx; i++) {
            const int32_t q[4] = {pid(i, ny, k), pid(i, ny, k + 1), pid(i + 1, ny, k + 1), pid(i + 1, ny, k)};
            push(cid(i, ny - 1, k), q);
        }
    for (int j = 0; j < ny; j++)  // z-min
        for (int i = 0; i < nx; i++) {
            const int32_t q[4] = {pid(i, j, 0), pid(i, j + 1, 0), pid(i + 1, j + 1, 0), pid(i + 1, j, 0)};
            push(cid(i, j, 0), q);
        }
    for (int j = 0; j < ny; j++)  // z-max
        for (int i = 0; i < nx; i++) {
            const int32_t q[4] = {pid(i, j, nz), pid(i + 1, j, nz), pid(i + 1, j + 1, nz), pid(i, j + 1, nz)};
            push(cid(i, j, nz - 1), q);
        }
}

}  // namespace

extern "C" {

int jfnk_hex_patch(int nx, int ny, int nz, int side, int32_t* first_face, int32_t* n_faces)
{
    if (nx < 1 || ny < 1 || nz < 1 || side < 0 || side > 5) return JFNK_EINVAL;
    const int64_t sizes[6] = {(int64_t)ny * nz, (int64_t)ny * nz, (int64_t)nx * nz, (int64_t)nx * nz,
                              (int64_t)nx * ny, (int64_t)nx * ny};
    int64_t first = n_internal_faces(nx, ny, nz);
    for (int s = 0; s < side; s++) first += sizes[s];
    if (first + sizes[side] > INT32_MAX) return JFNK_EINVAL;
    if (first_face) *first_face = (int32_t)first;
    if (n_faces) *n_faces = (int32_t)sizes[side];
    return JFNK_OK;
}

int jfnk_set_mesh_hex(jfnk_ctx* ctx, int nx, int ny, int nz, const double* points, int dim)
{
    if (!ctx) return JFNK_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || !points || (dim != 2 && dim != 3) || (dim == 2 && nz != 1)) return JFNK_EINVAL;
    const int64_t ncells = (int64_t)nx * ny * nz, npts = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    const int64_t nfaces = n_internal_faces(nx, ny, nz) + 2 * ((int64_t)ny * nz + (int64_t)nx * nz + (int64_t)nx * ny);
    if (4 * nfaces > INT32_MAX || npts > INT32_MAX) return JFNK_EINVAL;
    HexFaces h;
    build(nx, ny, nz, h);
    int rc = jfnk_set_mesh(ctx, dim, (int32_t)npts, points, (int32_t)nfaces, h.ptr.data(), h.pts.data(), h.own.data(),
                           (int32_t)h.nei.size(), h.nei.data(), (int32_t)ncells);
    if (rc || dim == 3) return rc;
    for (int side = 4; side < 6; side++) {
        int32_t f0 = 0, nf = 0;
        jfnk_hex_patch(nx, ny, nz, side, &f0, &nf);
        if ((rc = jfnk_set_patch(ctx, f0, nf, JFNK_BC_EMPTY, nullptr))) return rc;
    }
    return JFNK_OK;
}

}  // extern "C"
