// The paper's own outer-volume estimator (Sec. 4.1, Eq. 9-10), restated as
// CUDA ray casting instead of cube-map rasterisation.
//
// From the box centre o, one ray per texel of a 6 x m x m cube map (direction
// through the texel centre, weight = the texel's exact solid angle).  Along a
// ray the mesh crossings at distances r_i < r_e (r_e = where the ray leaves the
// box) carry sign s_i = +1 when the ray leaves the solid (n . w > 0) and -1
// when it enters (the convention of Fig. 1a).  With chi(o) = 1 when o is
// inside the solid, the inside length of the segment is
//   l_in = sum_i s_i r_i + chi(p_e) r_e,   chi(p_e) = chi(o) - sum_i s_i,
// and the cone volumes give
//   V_out(w) = dOmega / 3 (r_e^3 - sum_i s_i r_i^3 - chi(p_e) r_e^3).
// The estimate is the sum over texels.  chi(o) is the signed crossing count of
// a ray from o to infinity (outward-oriented closed mesh).  FP32 arithmetic,
// Moeller-Trumbore intersections against every triangle.
#include "internal.h"

namespace obbv {
namespace {

__device__ __forceinline__ bool ray_tri(const float3 o, const float3 d, const float3 a, const float3 b,
                                        const float3 c, float& t, float& sgn)
{
    const float3 e1 = make_float3(b.x - a.x, b.y - a.y, b.z - a.z);
    const float3 e2 = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
    const float3 p = make_float3(d.y * e2.z - d.z * e2.y, d.z * e2.x - d.x * e2.z, d.x * e2.y - d.y * e2.x);
    const float det = e1.x * p.x + e1.y * p.y + e1.z * p.z;
    if (fabsf(det) < 1e-20f) return false;
    const float inv = 1.f / det;
    const float3 s = make_float3(o.x - a.x, o.y - a.y, o.z - a.z);
    const float u = (s.x * p.x + s.y * p.y + s.z * p.z) * inv;
    if (u < 0.f || u > 1.f) return false;
    const float3 q = make_float3(s.y * e1.z - s.z * e1.y, s.z * e1.x - s.x * e1.z, s.x * e1.y - s.y * e1.x);
    const float v = (d.x * q.x + d.y * q.y + d.z * q.z) * inv;
    if (v < 0.f || u + v > 1.f) return false;
    t = (e2.x * q.x + e2.y * q.y + e2.z * q.z) * inv;
    if (t <= 0.f) return false;
    // outward normal e1 x e2: leaving the solid when it points along d (det = -(e1 x e2) . d)
    sgn = det < 0.f ? 1.f : -1.f;
    return true;
}

__device__ __forceinline__ float texel_solid_angle(float u0, float u1, float v0, float v1)
{
    auto F = [](float u, float v) { return atan2f(u * v, sqrtf(u * u + v * v + 1.f)); };
    return F(u1, v1) - F(u0, v1) - F(u1, v0) + F(u0, v0);
}

// one block per box; threads stride over the 6 m^2 texels
__global__ void k_directional(const float* __restrict__ V, const int32_t* __restrict__ Fi, int64_t nt,
                              const obb_box* __restrict__ boxes, int32_t m, double* __restrict__ out)
{
    const obb_box B = boxes[blockIdx.x];
    const float3 o = make_float3(B.c[0], B.c[1], B.c[2]);
    const float3 ax[3] = {make_float3(B.axis0[0], B.axis0[1], B.axis0[2]),
                          make_float3(B.axis1[0], B.axis1[1], B.axis1[2]),
                          make_float3(B.axis0[1] * B.axis1[2] - B.axis0[2] * B.axis1[1],
                                      B.axis0[2] * B.axis1[0] - B.axis0[0] * B.axis1[2],
                                      B.axis0[0] * B.axis1[1] - B.axis0[1] * B.axis1[0])};
    // chi(o): signed crossings of a ray from o towards a fixed generic direction
    __shared__ float chi;
    if (threadIdx.x == 0) chi = 0.f;
    __syncthreads();
    {
        const float3 d = make_float3(0.5773502f, 0.5773503f, 0.5773502f);
        float acc = 0.f;
        for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
            const float* a = V + 3 * (int64_t)Fi[3 * t];
            const float* b = V + 3 * (int64_t)Fi[3 * t + 1];
            const float* c = V + 3 * (int64_t)Fi[3 * t + 2];
            float tt, sg;
            if (ray_tri(o, d, make_float3(a[0], a[1], a[2]), make_float3(b[0], b[1], b[2]),
                        make_float3(c[0], c[1], c[2]), tt, sg))
                acc += sg;
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(&chi, acc);
    }
    __syncthreads();
    const float chi_o = rintf(chi);
    double vol = 0.0;
    const int texels = 6 * m * m;
    for (int x = threadIdx.x; x < texels; x += blockDim.x) {
        const int face = x / (m * m), r = x % (m * m), iu = r % m, iv = r / m;
        const float u0 = -1.f + 2.f * iu / m, u1 = -1.f + 2.f * (iu + 1) / m;
        const float v0 = -1.f + 2.f * iv / m, v1 = -1.f + 2.f * (iv + 1) / m;
        const float uc = 0.5f * (u0 + u1), vc = 0.5f * (v0 + v1);
        float3 d;
        const int axis = face >> 1;
        const float sgn = (face & 1) ? -1.f : 1.f;
        float w[3];
        w[axis] = sgn;
        w[(axis + 1) % 3] = uc;
        w[(axis + 2) % 3] = vc;
        const float nrm = rsqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        d = make_float3(w[0] * nrm, w[1] * nrm, w[2] * nrm);
        // exit distance from the box (centre o): min_a half_a / |axis_a . d|
        float re = 3.0e38f;
        for (int a = 0; a < 3; ++a) {
            const float c = fabsf(ax[a].x * d.x + ax[a].y * d.y + ax[a].z * d.z);
            if (c > 0.f) re = fminf(re, B.half[a] / c);
        }
        float s1 = 0.f, s3 = 0.f;
        for (int64_t t = 0; t < nt; ++t) {
            const float* a = V + 3 * (int64_t)Fi[3 * t];
            const float* b = V + 3 * (int64_t)Fi[3 * t + 1];
            const float* c = V + 3 * (int64_t)Fi[3 * t + 2];
            float tt, sg;
            if (ray_tri(o, d, make_float3(a[0], a[1], a[2]), make_float3(b[0], b[1], b[2]),
                        make_float3(c[0], c[1], c[2]), tt, sg) &&
                tt < re) {
                s1 += sg;
                s3 += sg * tt * tt * tt;
            }
        }
        const float chi_e = chi_o - s1;
        const float re3 = re * re * re;
        vol += (double)texel_solid_angle(u0, u1, v0, v1) / 3.0 * ((double)re3 - s3 - chi_e * re3);
    }
    for (int off = 16; off > 0; off >>= 1) vol += __shfl_xor_sync(0xffffffffu, vol, off);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = vol;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += part[i];
        out[blockIdx.x] = tot;
    }
}

}  // namespace

obb_status directional_outer_volume(obb_ctx* ctx, const obb_mesh* mesh, const obb_box* d_boxes, int64_t K, int32_t m,
                                    double* d_out)
{
    if (K <= 0) return OBB_OK;
    k_directional<<<(unsigned)K, 256, 0, ctx->stream>>>(mesh->d_verts, mesh->d_tris, mesh->nt, d_boxes, m, d_out);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

}  // namespace obbv
