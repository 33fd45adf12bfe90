// adjoint.cu -- gradient of the per-cell moments (volume V_i, centroid c_i,
// second moment M2_i = integral over C_i of |x - p_i|^2) with respect to
// the generators, for Lloyd relaxation and other losses of the cells.
//
// For upstream gradients (gV_i, gC_i, gM_i) cell i carries the density
//     h_i(x) = gV_i + gC_i . (x - c_i) / V_i + gM_i |x - p_i|^2
// and grad_k = 2 gM_k V_k (p_k - c_k)                                (interior)
//            + sum over faces f of cell k, neighbour j, d = |p_j - p_k|:
//                (1/d) integral_f h_k(x) (x - p_k) dA               (face of k moves with p_k)
//              + (1/d) integral_f h_j(x) (p_k - x) dA               (face of j moves with p_k)
// (a face on the bisector moves along its normal with speed (x - p_k).dp_k / d
// seen from cell k and (p_k - x).dp_k / d seen from cell j; walls are fixed).
//
// Everything is integrated in the frame of p_k (y = x - p_k). On the shared
// face |x - p_j| = |x - p_k| = |y|, so both densities read a + b.y + g |y|^2
// there (each density's constant absorbs b.(p_k - c)), and one set of face
// moments -- M1, M2, Q1 of y, y y^T, |y|^2 y -- serves both.
// The moments are integrated exactly on the face's triangle fan with the
// 7-point degree-3 rule. Gather form: one warp per cell sums every
// contribution to its own generator (deterministic, no atomics). The face
// integrals run in the precision of the tessellation (float32 for the FP32
// form: the FP64 rate of the part is 1/64 of float32; the local frame keeps
// the values small), the per-cell sums across lanes in FP64.
//
// Periodic box: the neighbour across a face is an image p_j + t L. The face
// lies on the bisector of p_k and that image, so the image is the reflection
// of p_k across the face's plane; t is that reflection minus p_j over L,
// rounded (the plane comes from the face's own vertices: its area vector
// and its first vertex). Cell j's density is then read through the same
// image (its centroid shifted by t L).
#include "vt_internal.cuh"

namespace vt {

namespace {

template <typename Real>
struct Dens {
    Real a, bx, by, bz, g;  // h(y) = a + b.y + g |y|^2 in the frame of p_k
};

// density of cell i written in the frame of the point (px, py, pz)
template <typename Real>
__device__ __forceinline__ Dens<Real> density(int i, double px, double py, double pz, const double* vol,
                                              const double* cen, const double* gV, const double* gC, const double* gM)
{
    Dens<Real> d;
    d.g = (Real)(gM ? gM[i] : 0.0);
    d.bx = d.by = d.bz = (Real)0;
    d.a = (Real)(gV ? gV[i] : 0.0);
    if (gC) {  // gV + b.(x - c) with x = y + p, b = gC / V
        const Real V = (Real)vol[i];
        d.bx = (Real)gC[3 * i] / V;
        d.by = (Real)gC[3 * i + 1] / V;
        d.bz = (Real)gC[3 * i + 2] / V;
        d.a += d.bx * (Real)(px - cen[3 * i]) + d.by * (Real)(py - cen[3 * i + 1]) + d.bz * (Real)(pz - cen[3 * i + 2]);
    }
    return d;
}

// integral over the face of h y, from the face moments
template <typename Real>
__device__ __forceinline__ void face_term(const Dens<Real>& h, const Real* M1, const Real* M2, const Real* Q1,
                                          Real* out)
{
    out[0] = h.a * M1[0] + M2[0] * h.bx + M2[1] * h.by + M2[2] * h.bz + h.g * Q1[0];
    out[1] = h.a * M1[1] + M2[1] * h.bx + M2[3] * h.by + M2[4] * h.bz + h.g * Q1[1];
    out[2] = h.a * M1[2] + M2[2] * h.bx + M2[4] * h.by + M2[5] * h.bz + h.g * Q1[2];
}

template <typename Real>
__global__ void __launch_bounds__(256) k_adjoint(const float* __restrict__ pts, int64_t n,
                                                 const double* __restrict__ vol, const double* __restrict__ cen,
                                                 const int64_t* __restrict__ vtx_off, const double* __restrict__ vtx,
                                                 const int64_t* __restrict__ face_off,
                                                 const int32_t* __restrict__ face_nbr,
                                                 const int64_t* __restrict__ face_vtx_off,
                                                 const int32_t* __restrict__ face_vtx, const double* __restrict__ gV,
                                                 const double* __restrict__ gC, const double* __restrict__ gM,
                                                 double* __restrict__ grad, const __grid_constant__ GridDesc box)
{
    const bool per = box.periodic != 0;
    const double Lx = (double)box.hi[0] - (double)box.lo[0], Ly = (double)box.hi[1] - (double)box.lo[1],
                 Lz = (double)box.hi[2] - (double)box.lo[2];
    // 7-point degree-3 rule: vertices 1/20, edge midpoints 2/15, centroid 9/20
    const Real wv = (Real)(1.0 / 20.0), we = (Real)(2.0 / 15.0), wc = (Real)(9.0 / 20.0);
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = wid; k < n; k += nw) {
        const double px = pts[3 * k], py = pts[3 * k + 1], pz = pts[3 * k + 2];
        const Dens<Real> hk = density<Real>((int)k, px, py, pz, vol, cen, gV, gC, gM);
        const double* V = vtx + 3 * vtx_off[k];
        Real gx = 0, gy = 0, gz = 0;
        const int64_t f0 = face_off[k], f1 = face_off[k + 1];
        for (int64_t f = f0 + lane; f < f1; f += 32) {
            const int j = face_nbr[f];
            if (j < 0) continue;  // walls do not move
            Real M1[3] = {0, 0, 0}, M2[6] = {0, 0, 0, 0, 0, 0}, Q1[3] = {0, 0, 0};
            const int32_t* loop = face_vtx + face_vtx_off[f];
            const int deg = (int)(face_vtx_off[f + 1] - face_vtx_off[f]);
            // vertices in the frame of p_k
            const double* A0 = V + 3 * loop[0];
            const Real A[3] = {(Real)(A0[0] - px), (Real)(A0[1] - py), (Real)(A0[2] - pz)};
            const double* B0 = V + 3 * loop[1];
            Real B[3] = {(Real)(B0[0] - px), (Real)(B0[1] - py), (Real)(B0[2] - pz)};
            Real sx = 0, sy = 0, sz = 0;  // twice the face's area vector (outward)
            for (int t = 1; t + 1 < deg; ++t) {
                const double* C0 = V + 3 * loop[t + 1];
                const Real C[3] = {(Real)(C0[0] - px), (Real)(C0[1] - py), (Real)(C0[2] - pz)};
                const Real ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
                const Real vx = C[0] - A[0], vy = C[1] - A[1], vz = C[2] - A[2];
                const Real cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
                const Real area = (Real)0.5 * sqrt(cx * cx + cy * cy + cz * cz);
                sx += cx;
                sy += cy;
                sz += cz;
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    // barycentric point q of the rule
                    Real l0, l1, l2, w;
                    if (q < 3) { l0 = q == 0; l1 = q == 1; l2 = q == 2; w = wv; }
                    else if (q < 6) { l0 = q != 4 ? (Real)0.5 : (Real)0; l1 = q != 5 ? (Real)0.5 : (Real)0; l2 = q != 3 ? (Real)0.5 : (Real)0; w = we; }
                    else { l0 = l1 = l2 = (Real)(1.0 / 3.0); w = wc; }
                    const Real x = l0 * A[0] + l1 * B[0] + l2 * C[0];
                    const Real y = l0 * A[1] + l1 * B[1] + l2 * C[1];
                    const Real z = l0 * A[2] + l1 * B[2] + l2 * C[2];
                    const Real wa = w * area;
                    const Real qq = x * x + y * y + z * z;
                    M1[0] += wa * x; M1[1] += wa * y; M1[2] += wa * z;
                    M2[0] += wa * x * x; M2[1] += wa * x * y; M2[2] += wa * x * z;
                    M2[3] += wa * y * y; M2[4] += wa * y * z; M2[5] += wa * z * z;
                    Q1[0] += wa * qq * x; Q1[1] += wa * qq * y; Q1[2] += wa * qq * z;
                }
                B[0] = C[0]; B[1] = C[1]; B[2] = C[2];
            }
            double ox = 0.0, oy = 0.0, oz = 0.0;  // t L of the image across the face
            if (per) {
                // reflection of p_k across the face plane: 2 (n.A) n, n the unit normal
                const double sn = sqrt((double)sx * sx + (double)sy * sy + (double)sz * sz);
                if (sn > 0.0) {
                    const double nx = sx / sn, ny = sy / sn, nz = sz / sn;
                    const double h2 = 2.0 * (nx * (double)A[0] + ny * (double)A[1] + nz * (double)A[2]);
                    ox = rint((px + h2 * nx - (double)pts[3 * (int64_t)j]) / Lx) * Lx;
                    oy = rint((py + h2 * ny - (double)pts[3 * (int64_t)j + 1]) / Ly) * Ly;
                    oz = rint((pz + h2 * nz - (double)pts[3 * (int64_t)j + 2]) / Lz) * Lz;
                }
            }
            const Real dx = (Real)(((double)pts[3 * (int64_t)j] - px) + ox),
                       dy = (Real)(((double)pts[3 * (int64_t)j + 1] - py) + oy),
                       dz = (Real)(((double)pts[3 * (int64_t)j + 2] - pz) + oz);
            const Real inv_d = (Real)1 / sqrt(dx * dx + dy * dy + dz * dz);
            // cell j seen through its image: its density in the frame of p_k - t L
            const Dens<Real> hj = density<Real>(j, px - ox, py - oy, pz - oz, vol, cen, gV, gC, gM);
            Real own[3], nbr[3];
            face_term(hk, M1, M2, Q1, own);  // integral of h_k y
            face_term(hj, M1, M2, Q1, nbr);  // integral of h_j y
            gx += (own[0] - nbr[0]) * inv_d;
            gy += (own[1] - nbr[1]) * inv_d;
            gz += (own[2] - nbr[2]) * inv_d;
        }
        double sx = (double)gx, sy = (double)gy, sz = (double)gz;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        if (lane == 0) {
            const double s = 2.0 * (gM ? gM[k] : 0.0) * vol[k];  // interior term of M2: 2 gM V (p - c)
            grad[3 * k] = sx + s * (px - cen[3 * k]);
            grad[3 * k + 1] = sy + s * (py - cen[3 * k + 1]);
            grad[3 * k + 2] = sz + s * (pz - cen[3 * k + 2]);
        }
    }
}

// Lloyd's update written as a gradient step on the energy sum_i M2_i:
// p <- p - g / (2 V) with g = d(sum M2)/dp = 2 V (p - c), which lands on the
// centroid (Lloyd 1982), in FP64 and rounded once to float32. In a periodic
// box the new point is moved by whole periods into [lo, hi) (in FP64 from the
// rounded value, rounded again; a value that rounds onto hi belongs at lo);
// in a walled box a value that rounds onto hi is moved to the largest float
// below it, so the next tessellation gets a valid point.
__global__ void k_lloyd_step(const float* __restrict__ pts, int64_t n, const double* __restrict__ grad,
                             const double* __restrict__ vol, GridDesc g, float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / 3;
        const int a = (int)(i - 3 * k);
        const double lo = (double)g.lo[a], hi = (double)g.hi[a];
        float x = (float)((double)pts[i] - grad[i] / (2.0 * vol[k]));
        if (g.periodic) {
            const double L = hi - lo, xd = (double)x;
            x = (float)(xd - floor((xd - lo) / L) * L);
            if (x >= g.hi[a]) x = g.lo[a];
        } else if (x >= g.hi[a]) {
            x = nextafterf(g.hi[a], g.lo[a]);
        }
        out[i] = x;
    }
}

}  // namespace

cudaError_t launch_lloyd_step(const float* pts, int64_t n, const double* grad, const double* vol, const GridDesc& g,
                              float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (3 * n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_lloyd_step<<<(unsigned)blocks, 256, 0, s>>>(pts, n, grad, vol, g, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const float* pts, int64_t n, const vt_cells_out& c, const double* gV, const double* gC,
                           const double* gM, double* grad, int precision, const GridDesc& g, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 7) / 8;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (precision == VT_FP64)
        k_adjoint<double><<<(unsigned)blocks, 256, 0, s>>>(pts, n, c.vol, c.cen, c.vtx_off, c.vtx, c.face_off,
                                                           c.face_nbr, c.face_vtx_off, c.face_vtx, gV, gC, gM, grad, g);
    else
        k_adjoint<float><<<(unsigned)blocks, 256, 0, s>>>(pts, n, c.vol, c.cen, c.vtx_off, c.vtx, c.face_off,
                                                          c.face_nbr, c.face_vtx_off, c.face_vtx, gV, gC, gM, grad, g);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vt
