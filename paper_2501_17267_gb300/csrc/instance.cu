// instance.cu -- tile-planting instance generator (host) and instance handles.
//
// Tile planting (arXiv:2501.17267, Sec. II): the periodic lattice is cut into unit
// cubes ("tiles") whose origins have all-even or all-odd coordinates; these N/4
// cubes share no edge and cover every edge once.  Each tile takes the couplings of
// a class template placed under a random cube symmetry.  Each template has the
// all-+1 corner state among its ground states, so the global all-+1 state is a
// ground state of the whole lattice and E_gs is the sum of the template minima.
// A random gauge tau then hides it: J'_ij = J_ij tau_i tau_j, planted state tau.
//
// The class templates are ferromagnetic cubes (J = -1) with a few antiferromagnetic
// (J = +1) edges that frustrate the faces the class is named after:
//   F22: x-edge at corner (0,0,0)                               -> 2 adjacent faces
//   F42: x-edges at (0,0,0) and (0,1,1)                         -> 4 faces, x-faces free
//   F6 : x-edge at (0,0,0), y-edge at (0,0,1), z-edge at (1,1,0) -> all 6 faces
// with minima -10, -8, -6 (one, two, three unsatisfiable edges).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>

#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

struct TemplateEdge {
    int corner[3];  // lower corner of the edge inside the unit cube
    int axis;       // 0 = x, 1 = y, 2 = z
    int8_t J;
};

// The twelve edges of a class template, each with its coupling.
std::array<TemplateEdge, 12> class_template(int cls)
{
    std::array<TemplateEdge, 12> t{};
    int n = 0;
    for (int axis = 0; axis < 3; ++axis)
        for (int hi = 0; hi < 2; ++hi)
            for (int lo = 0; lo < 2; ++lo) {
                // the two coordinates other than `axis`, lower axis first
                int c[3] = {0, 0, 0};
                int oa = axis == 0 ? 1 : 0;
                int ob = axis == 2 ? 1 : 2;
                c[oa] = lo;
                c[ob] = hi;
                t[n].corner[0] = c[0];
                t[n].corner[1] = c[1];
                t[n].corner[2] = c[2];
                t[n].axis = axis;
                t[n].J = -1;
                ++n;
            }
    auto flip = [&](int axis, int x, int y, int z) {
        for (auto& e : t)
            if (e.axis == axis && e.corner[0] == x && e.corner[1] == y && e.corner[2] == z)
                e.J = +1;
    };
    flip(0, 0, 0, 0);
    if (cls == 1) flip(0, 0, 1, 1);
    if (cls == 2) {
        flip(1, 0, 0, 1);
        flip(2, 1, 1, 0);
    }
    return t;
}

constexpr int kTemplateMin[3] = {-10, -8, -6};

// Cube symmetry g = 8 p + r: axis permutation p (lexicographic order over the six
// permutations of (x, y, z)) and reflection bits r.  The image of a corner has, on
// axis a, the original coordinate on axis perm[a], mirrored when bit a of r is set.
struct CubeSymmetry {
    int perm[3];
    int refl;
    void apply(const int in[3], int out[3]) const
    {
        for (int a = 0; a < 3; ++a) out[a] = in[perm[a]] ^ ((refl >> a) & 1);
    }
};

CubeSymmetry cube_symmetry(int g)
{
    int perms[6][3];
    int order[3] = {0, 1, 2};
    int n = 0;
    do {
        perms[n][0] = order[0];
        perms[n][1] = order[1];
        perms[n][2] = order[2];
        ++n;
    } while (std::next_permutation(order, order + 3));
    CubeSymmetry s;
    for (int a = 0; a < 3; ++a) s.perm[a] = perms[g / 8][a];
    s.refl = g % 8;
    return s;
}

struct PlacedEdge {  // tile-relative lower corner and axis of an image edge
    int dx, dy, dz, axis;
    int8_t J;
};

}  // namespace

int32_t generate_instance(int L, uint64_t seed, const double class_prob[3], int gauge,
                          int8_t* J3, int8_t* planted, int64_t* e_gs)
{
    if (L < 2 || L > SG_LMAX || (L & 1)) {
        set_error("L must be even with 2 <= L <= %d (got %d)", SG_LMAX, L);
        return SG_EINVAL;
    }
    const double w0 = class_prob[0], w1 = class_prob[1], w2 = class_prob[2];
    if (!(w0 >= 0 && w1 >= 0 && w2 >= 0) || !(w0 + w1 + w2 > 0)) {
        set_error("class_prob must be non-negative with a positive sum");
        return SG_EINVAL;
    }
    const double total = w0 + w1 + w2;
    // inverse CDF of a 32-bit uniform word against cumulative weights in 2^32 fixed point
    const uint64_t cut0 = (uint64_t)floor(ldexp(w0 / total, 32));
    const uint64_t cut1 = (uint64_t)floor(ldexp((w0 + w1) / total, 32));

    // all (class, symmetry) placements, precomputed
    static std::array<std::array<std::array<PlacedEdge, 12>, 48>, 3> placed = [] {
        std::array<std::array<std::array<PlacedEdge, 12>, 48>, 3> P{};
        for (int cls = 0; cls < 3; ++cls) {
            auto t = class_template(cls);
            for (int g = 0; g < 48; ++g) {
                CubeSymmetry s = cube_symmetry(g);
                for (int e = 0; e < 12; ++e) {
                    int a[3] = {t[e].corner[0], t[e].corner[1], t[e].corner[2]};
                    int b[3] = {a[0], a[1], a[2]};
                    b[t[e].axis] = 1;
                    int ga[3], gb[3];
                    s.apply(a, ga);
                    s.apply(b, gb);
                    int axis = 0;
                    while (ga[axis] == gb[axis]) ++axis;
                    const int* lo = ga[axis] < gb[axis] ? ga : gb;
                    P[cls][g][e] = PlacedEdge{lo[0], lo[1], lo[2], axis, t[e].J};
                }
            }
        }
        return P;
    }();

    const int64_t N = (int64_t)L * L * L;
    const int H = L / 2;
    const int64_t half = (int64_t)H * H * H;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    auto wrap = [L](int v) { return v >= L ? v - L : v; };
    int64_t E = 0;
    for (int parity = 0; parity < 2; ++parity)
        for (int c = 0; c < H; ++c)
            for (int b = 0; b < H; ++b)
                for (int a = 0; a < H; ++a) {
                    const int64_t t = parity * half + a + (int64_t)H * (b + (int64_t)H * c);
                    const Philox4 r = philox4x32_10((uint32_t)t, 0, 0, kDomainGenerate, k0, k1);
                    const int cls = r.v[0] < cut0 ? 0 : (r.v[0] < cut1 ? 1 : 2);
                    const int g = (int)(((uint64_t)r.v[1] * 48u) >> 32);
                    E += kTemplateMin[cls];
                    const int ox = 2 * a + parity, oy = 2 * b + parity, oz = 2 * c + parity;
                    for (const PlacedEdge& pe : placed[cls][g]) {
                        const int64_t i = wrap(ox + pe.dx) +
                                          (int64_t)L * (wrap(oy + pe.dy) + (int64_t)L * wrap(oz + pe.dz));
                        J3[3 * i + pe.axis] = pe.J;
                    }
                }
    for (int64_t i = 0; i < N; ++i) {
        const Philox4 r = philox4x32_10((uint32_t)i, 0, 0, kDomainGauge, k0, k1);
        planted[i] = (gauge && (r.v[0] >> 31)) ? -1 : 1;
    }
    if (gauge) {
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    const int64_t i = x + (int64_t)L * (y + (int64_t)L * z);
                    const int64_t nb[3] = {wrap(x + 1) + (int64_t)L * (y + (int64_t)L * z),
                                           x + (int64_t)L * (wrap(y + 1) + (int64_t)L * z),
                                           x + (int64_t)L * (y + (int64_t)L * wrap(z + 1))};
                    for (int d = 0; d < 3; ++d)
                        J3[3 * i + d] = (int8_t)(J3[3 * i + d] * planted[i] * planted[nb[d]]);
                }
    }
    *e_gs = E;
    return SG_OK;
}

// Upload J3 and build the per-site six-coupling records on the current device
// (once per device; later calls reuse the copy).
int32_t instance_device_j6(sg_instance* inst, cudaStream_t stream, const uint2** j6,
                           const uint8_t** j1)
{
    int dev = 0;
    SG_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(inst->mu);
    for (auto& d : inst->dev)
        if (d.device == dev) {
            *j6 = d.j6;
            if (j1) *j1 = d.j1;
            return SG_OK;
        }
    DeviceCopy dc;
    dc.device = dev;
    int8_t* J3d = nullptr;
    const size_t N = (size_t)inst->N;
    // one allocation: [N] uint2 records, then [N] sign bytes
    cudaError_t e = cudaMalloc(&dc.j6, sizeof(uint2) * N + N);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc: %s", cudaGetErrorString(e));
        return SG_ENOMEM;
    }
    dc.j1 = reinterpret_cast<uint8_t*>(dc.j6 + N);
    e = cudaMalloc(&J3d, 3 * N);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dc.j6);
        set_error("cudaMalloc: %s", cudaGetErrorString(e));
        return SG_ENOMEM;
    }
    e = cudaMemcpyAsync(J3d, inst->J3.data(), 3 * N, cudaMemcpyHostToDevice, stream);
    int32_t rc = e == cudaSuccess ? launch_prepare_j6(J3d, dc.j6, dc.j1, inst->L, stream) : SG_ECUDA;
    if (rc == SG_OK) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) rc = SG_ECUDA;
    }
    cudaFree(J3d);
    if (rc != SG_OK) {
        cudaFree(dc.j6);
        set_error("uploading couplings failed: %s", cudaGetErrorString(e));
        return rc;
    }
    inst->dev.push_back(dc);
    *j6 = dc.j6;
    if (j1) *j1 = dc.j1;
    return SG_OK;
}

}  // namespace sg

using namespace sg;

static int32_t finish_instance(sg_instance* inst)
{
    int64_t s = 0;
    bool unit = true;
    for (int8_t j : inst->J3) {
        s += j < 0 ? -j : j;
        unit &= (j == 1 || j == -1);
    }
    inst->abs_sum = (int32_t)s;
    inst->unit_couplings = unit;
    return SG_OK;
}

extern "C" int32_t sg_instance_create(const sg_instance_desc* d, sg_instance** out)
{
    clear_error();
    if (!d || !out) {
        set_error("NULL argument");
        return SG_EINVAL;
    }
    if (d->L < 2 || d->L > SG_LMAX || (d->L & 1)) {
        set_error("L must be even with 2 <= L <= %d (got %d)", SG_LMAX, d->L);
        return SG_EINVAL;
    }
    sg_instance* inst = new (std::nothrow) sg_instance;
    if (!inst) return SG_ENOMEM;
    inst->L = d->L;
    inst->N = (int64_t)d->L * d->L * d->L;
    try {
        inst->J3.assign((size_t)(3 * inst->N), 0);
        inst->planted.assign((size_t)inst->N, 1);
    } catch (...) {
        delete inst;
        set_error("host allocation failed");
        return SG_ENOMEM;
    }
    int32_t rc = generate_instance(d->L, d->seed, d->class_prob, d->gauge, inst->J3.data(),
                                   inst->planted.data(), &inst->e_gs);
    if (rc != SG_OK) {
        delete inst;
        return rc;
    }
    finish_instance(inst);
    *out = inst;
    return SG_OK;
}

extern "C" int32_t sg_instance_create_from_couplings(int32_t L, const int8_t* J3, int32_t mem_kind,
                                                     int64_t e_gs, sg_instance** out)
{
    clear_error();
    if (!J3 || !out || (mem_kind != SG_MEM_HOST && mem_kind != SG_MEM_DEVICE)) {
        set_error("NULL argument or bad mem_kind");
        return SG_EINVAL;
    }
    if (L < 2 || L > SG_LMAX || (L & 1)) {
        set_error("L must be even with 2 <= L <= %d (got %d)", SG_LMAX, L);
        return SG_EINVAL;
    }
    sg_instance* inst = new (std::nothrow) sg_instance;
    if (!inst) return SG_ENOMEM;
    inst->L = L;
    inst->N = (int64_t)L * L * L;
    inst->e_gs = e_gs;
    try {
        inst->J3.resize((size_t)(3 * inst->N));
        inst->planted.assign((size_t)inst->N, 1);
    } catch (...) {
        delete inst;
        set_error("host allocation failed");
        return SG_ENOMEM;
    }
    if (mem_kind == SG_MEM_DEVICE) {
        cudaError_t e = cudaMemcpy(inst->J3.data(), J3, inst->J3.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            delete inst;
            set_error("cudaMemcpy: %s", cudaGetErrorString(e));
            return SG_ECUDA;
        }
    } else {
        memcpy(inst->J3.data(), J3, inst->J3.size());
    }
    for (int8_t j : inst->J3)
        if (j > SG_JMAX || j < -SG_JMAX) {
            delete inst;
            set_error("coupling %d exceeds |J| <= %d", (int)j, SG_JMAX);
            return SG_EINVAL;
        }
    finish_instance(inst);
    *out = inst;
    return SG_OK;
}

extern "C" int32_t sg_instance_get(const sg_instance* inst, int32_t* L_out, int8_t* J3_out,
                                   int8_t* planted_out, int64_t* e_gs_out)
{
    clear_error();
    if (!inst) {
        set_error("NULL instance");
        return SG_EINVAL;
    }
    if (L_out) *L_out = inst->L;
    if (J3_out) memcpy(J3_out, inst->J3.data(), inst->J3.size());
    if (planted_out) memcpy(planted_out, inst->planted.data(), inst->planted.size());
    if (e_gs_out) *e_gs_out = inst->e_gs;
    return SG_OK;
}

extern "C" int32_t sg_instance_destroy(sg_instance* inst)
{
    clear_error();
    if (!inst) return SG_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& d : inst->dev) {
        cudaSetDevice(d.device);
        cudaFree(d.j6);
    }
    if (!inst->dev.empty()) cudaSetDevice(cur);
    delete inst;
    return SG_OK;
}
