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
// On the shared face |x - p_j| = |x - p_k|, so both densities are
// alpha + beta . x + gamma q(x) with q = |x - p_k|^2, and one set of face
// moments (M0, M1, M2, Q0, Q1 of 1, x, x x^T, q, q x) serves both. The moments
// are integrated exactly on the face's triangle fan with the 7-point
// degree-3 rule. Gather form: one warp per cell sums every contribution to
// its own generator in a fixed order (deterministic, no atomics), FP64.
#include "vt_internal.cuh"

namespace vt {

namespace {

struct Dens {
    double a, bx, by, bz, g;  // alpha, beta, gamma
};

__device__ __forceinline__ Dens density(int i, const double* vol, const double* cen, const double* gV,
                                        const double* gC, const double* gM)
{
    Dens d;
    const double V = vol[i];
    const double cx = cen[3 * i], cy = cen[3 * i + 1], cz = cen[3 * i + 2];
    d.bx = gC ? gC[3 * i] / V : 0.0;
    d.by = gC ? gC[3 * i + 1] / V : 0.0;
    d.bz = gC ? gC[3 * i + 2] / V : 0.0;
    d.a = (gV ? gV[i] : 0.0) - (d.bx * cx + d.by * cy + d.bz * cz);
    d.g = gM ? gM[i] : 0.0;
    return d;
}

// integral over the face of h (x - p): h = a + b.x + g q, from the face moments
__device__ __forceinline__ void face_term(const Dens& h, const double* M1, const double* M2, const double* Q1,
                                          double M0, double Q0, double px, double py, double pz, double* out)
{
    // integral of h x = a M1 + M2 b + g Q1; integral of h = a M0 + b.M1 + g Q0
    const double hx = h.a * M1[0] + M2[0] * h.bx + M2[1] * h.by + M2[2] * h.bz + h.g * Q1[0];
    const double hy = h.a * M1[1] + M2[1] * h.bx + M2[3] * h.by + M2[4] * h.bz + h.g * Q1[1];
    const double hz = h.a * M1[2] + M2[2] * h.bx + M2[4] * h.by + M2[5] * h.bz + h.g * Q1[2];
    const double h0 = h.a * M0 + h.bx * M1[0] + h.by * M1[1] + h.bz * M1[2] + h.g * Q0;
    out[0] = hx - px * h0;
    out[1] = hy - py * h0;
    out[2] = hz - pz * h0;
}

__global__ void __launch_bounds__(256) k_adjoint(const float* __restrict__ pts, int64_t n,
                                                 const double* __restrict__ vol, const double* __restrict__ cen,
                                                 const int64_t* __restrict__ vtx_off, const double* __restrict__ vtx,
                                                 const int64_t* __restrict__ face_off,
                                                 const int32_t* __restrict__ face_nbr,
                                                 const int64_t* __restrict__ face_vtx_off,
                                                 const int32_t* __restrict__ face_vtx, const double* __restrict__ gV,
                                                 const double* __restrict__ gC, const double* __restrict__ gM,
                                                 double* __restrict__ grad)
{
    // 7-point degree-3 rule: vertices 1/20, edge midpoints 2/15, centroid 9/20
    const double wv = 1.0 / 20.0, we = 2.0 / 15.0, wc = 9.0 / 20.0;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = wid; k < n; k += nw) {
        const double px = pts[3 * k], py = pts[3 * k + 1], pz = pts[3 * k + 2];
        const Dens hk = density((int)k, vol, cen, gV, gC, gM);
        const double* V = vtx + 3 * vtx_off[k];
        double gx = 0.0, gy = 0.0, gz = 0.0;
        const int64_t f0 = face_off[k], f1 = face_off[k + 1];
        for (int64_t f = f0 + lane; f < f1; f += 32) {
            const int j = face_nbr[f];
            if (j < 0) continue;  // walls do not move
            double M0 = 0, Q0 = 0, M1[3] = {0, 0, 0}, M2[6] = {0, 0, 0, 0, 0, 0}, Q1[3] = {0, 0, 0};
            const int32_t* loop = face_vtx + face_vtx_off[f];
            const int deg = (int)(face_vtx_off[f + 1] - face_vtx_off[f]);
            const double* A = V + 3 * loop[0];
            for (int t = 1; t + 1 < deg; ++t) {
                const double* B = V + 3 * loop[t];
                const double* C = V + 3 * loop[t + 1];
                const double ux = B[0] - A[0], uy = B[1] - A[1], uz = B[2] - A[2];
                const double vx = C[0] - A[0], vy = C[1] - A[1], vz = C[2] - A[2];
                const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
                const double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    // barycentric point q of the rule
                    double l0, l1, l2, w;
                    if (q < 3) { l0 = q == 0; l1 = q == 1; l2 = q == 2; w = wv; }
                    else if (q < 6) { l0 = q != 4 ? 0.5 : 0.0; l1 = q != 5 ? 0.5 : 0.0; l2 = q != 3 ? 0.5 : 0.0; w = we; }
                    else { l0 = l1 = l2 = 1.0 / 3.0; w = wc; }
                    const double x = l0 * A[0] + l1 * B[0] + l2 * C[0];
                    const double y = l0 * A[1] + l1 * B[1] + l2 * C[1];
                    const double z = l0 * A[2] + l1 * B[2] + l2 * C[2];
                    const double wa = w * area;
                    const double rx = x - px, ry = y - py, rz = z - pz;
                    const double qq = rx * rx + ry * ry + rz * rz;
                    M0 += wa;
                    M1[0] += wa * x; M1[1] += wa * y; M1[2] += wa * z;
                    M2[0] += wa * x * x; M2[1] += wa * x * y; M2[2] += wa * x * z;
                    M2[3] += wa * y * y; M2[4] += wa * y * z; M2[5] += wa * z * z;
                    Q0 += wa * qq;
                    Q1[0] += wa * qq * x; Q1[1] += wa * qq * y; Q1[2] += wa * qq * z;
                }
            }
            const double qx = pts[3 * (int64_t)j], qy = pts[3 * (int64_t)j + 1], qz = pts[3 * (int64_t)j + 2];
            const double dx = qx - px, dy = qy - py, dz = qz - pz;
            const double inv_d = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
            const Dens hj = density(j, vol, cen, gV, gC, gM);
            double own[3], nbr[3];
            face_term(hk, M1, M2, Q1, M0, Q0, px, py, pz, own);  // integral of h_k (x - p_k)
            face_term(hj, M1, M2, Q1, M0, Q0, px, py, pz, nbr);  // integral of h_j (x - p_k)
            gx += (own[0] - nbr[0]) * inv_d;
            gy += (own[1] - nbr[1]) * inv_d;
            gz += (own[2] - nbr[2]) * inv_d;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if (lane == 0) {
            const double s = 2.0 * hk.g * vol[k];  // interior term of M2: 2 gM V (p - c)
            grad[3 * k] = gx + s * (px - cen[3 * k]);
            grad[3 * k + 1] = gy + s * (py - cen[3 * k + 1]);
            grad[3 * k + 2] = gz + s * (pz - cen[3 * k + 2]);
        }
    }
}

}  // namespace

cudaError_t launch_adjoint(const float* pts, int64_t n, const vt_cells_out& c, const double* gV, const double* gC,
                           const double* gM, double* grad, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 7) / 8;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_adjoint<<<(unsigned)blocks, 256, 0, s>>>(pts, n, c.vol, c.cen, c.vtx_off, c.vtx, c.face_off, c.face_nbr,
                                               c.face_vtx_off, c.face_vtx, gV, gC, gM, grad);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vt
