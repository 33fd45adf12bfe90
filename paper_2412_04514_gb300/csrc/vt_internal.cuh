// vt_internal.cuh -- shared declarations of the CUDA path (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "vt.h"

namespace vt {

// ---------------------------------------------------------------------------
// grid description (host-computed, passed by value to kernels)
// ---------------------------------------------------------------------------
struct GridDesc {
    int G;            // cells per axis
    float lo[3];      // box
    float hi[3];
    float scale[3];   // float32(G) / (hi - lo), rounded once on the host
    double cw[3];     // cell width (hi - lo) / G in double (stop-rule geometry only)
    double margin;    // safety margin of the shell-walk stop rule (coordinates)
    int64_t cell_base;  // first global grid cell of this point set (batches)
    int64_t pt_begin;   // first input point of this point set
    int64_t npts;       // points in this point set
    int32_t periodic;   // 1: periodic box of periods hi - lo
    int32_t reserved;
};
static_assert(sizeof(GridDesc) == sizeof(vt_set_desc), "vt_set_desc mirrors GridDesc");

// grid of the point set that sorted point q belongs to
__device__ __forceinline__ const GridDesc& grid_of(const GridDesc& g0, const GridDesc* sets, const int32_t* set_of,
                                                   int q)
{
    return sets ? sets[set_of[q]] : g0;
}

// distance from q (in grid cell (ix, iy, iz)) to the outside of the block of
// shells 0..s, minus the rounding margin; FLT_MAX when the block reaches every
// wall of the box (no generator lies beyond it)
__device__ __forceinline__ float shell_gap(const GridDesc& g, float4 q, int ix, int iy, int iz, int s)
{
    // float32 throughout (the FP64 pipe is scarce): the grid's rounding
    // margin is taken twice, which also covers the float32 rounding of the
    // block bounds (a few ulps of the box extent)
    const int G = g.G;
    float gap = FLT_MAX;
    const float c0 = (float)g.cw[0], c1 = (float)g.cw[1], c2 = (float)g.cw[2];
    if (ix - s > 0) gap = fminf(gap, q.x - (g.lo[0] + (float)(ix - s) * c0));
    if (ix + s + 1 < G) gap = fminf(gap, (g.lo[0] + (float)(ix + s + 1) * c0) - q.x);
    if (iy - s > 0) gap = fminf(gap, q.y - (g.lo[1] + (float)(iy - s) * c1));
    if (iy + s + 1 < G) gap = fminf(gap, (g.lo[1] + (float)(iy + s + 1) * c1) - q.y);
    if (iz - s > 0) gap = fminf(gap, q.z - (g.lo[2] + (float)(iz - s) * c2));
    if (iz + s + 1 < G) gap = fminf(gap, (g.lo[2] + (float)(iz + s + 1) * c2) - q.z);
    return gap == FLT_MAX ? FLT_MAX : gap - 2.0f * (float)g.margin;
}

GridDesc make_grid(const vt_params* p, int G);

// grid cell of a point: every operation a separately rounded float32 op
__device__ __forceinline__ int cell_coord(float x, float lo, float scale, int G)
{
    float t = __fmul_rn(__fsub_rn(x, lo), scale);
    int c = (int)floorf(t);
    c = c < 0 ? 0 : c;
    return c > G - 1 ? G - 1 : c;
}

__device__ __forceinline__ int cell_id(int ix, int iy, int iz, int G) { return (ix * G + iy) * G + iz; }

// Segment e of Chebyshev shell s around grid cell (ix, iy, iz): a contiguous
// range [a, b) of the sorted points (empty when outside the grid). Row
// (dx, dy), dx, dy in [-s, s], owns segments 2*row and 2*row + 1: a row on the
// shell's rim (|dx| = s or |dy| = s) contributes the z-range [iz-s, iz+s] as
// its first segment; an inner row contributes the two cells z = iz-s and
// z = iz+s. A shell has 2 (2s+1)^2 segments, s = 0 has the cell itself.
__device__ __forceinline__ void shell_segment(int e, int s, int ix, int iy, int iz, int G,
                                              const int32_t* __restrict__ cell_off, int& a, int& b)
{
    const int W = 2 * s + 1;
    const int row = e >> 1, half = e & 1;
    const int dx = row / W - s, dy = row - (row / W) * W - s;
    const int x = ix + dx, y = iy + dy;
    a = b = 0;
    if (x < 0 || x >= G || y < 0 || y >= G) return;
    const bool rim = dx == -s || dx == s || dy == -s || dy == s;
    const int base = (x * G + y) * G;
    if (rim) {
        if (half) return;
        const int z0 = iz - s < 0 ? 0 : iz - s, z1 = iz + s > G - 1 ? G - 1 : iz + s;
        a = cell_off[base + z0];
        b = cell_off[base + z1 + 1];
    } else {
        const int z = half ? iz + s : iz - s;
        if (z < 0 || z >= G) return;
        a = cell_off[base + z];
        b = cell_off[base + z + 1];
    }
}

// The part of segment e of shell s (see shell_segment) whose grid cells reach
// into the ball of squared radius r_out2 around q and are not wholly inside
// the ball of squared radius r_in2 (r_in2 <= 0: none is skipped). A rim row's
// z-run loses its inner cells as two pieces: the part below is its first
// segment, the part above its second. Cell bounds are widened by the grid's
// rounding margin, so a cell is dropped only when no point assigned to it can
// lie in the annulus; callers pass radii that already carry their own margins.
__device__ __forceinline__ void shell_segment_ball(int e, int s, int ix, int iy, int iz, const GridDesc& g,
                                                   const int32_t* __restrict__ cell_off, float4 q, float r_out2,
                                                   float r_in2, int& a, int& b)
{
    const int G = g.G;
    const int W = 2 * s + 1;
    const int row = e >> 1, half = e & 1;
    const int dx = row / W - s, dy = row - (row / W) * W - s;
    const int x = ix + dx, y = iy + dy;
    a = b = 0;
    if (x < 0 || x >= G || y < 0 || y >= G) return;
    const float m = (float)g.margin;
    const float cx = (float)g.cw[0], cy = (float)g.cw[1], cz = (float)g.cw[2];
    const float x0 = g.lo[0] + (float)x * cx - m, x1 = g.lo[0] + (float)(x + 1) * cx + m;
    const float y0 = g.lo[1] + (float)y * cy - m, y1 = g.lo[1] + (float)(y + 1) * cy + m;
    const float dxn = fmaxf(fmaxf(x0 - q.x, q.x - x1), 0.0f), dyn = fmaxf(fmaxf(y0 - q.y, q.y - y1), 0.0f);
    const float dxf = fmaxf(q.x - x0, x1 - q.x), dyf = fmaxf(q.y - y0, y1 - q.y);
    const float dn2 = dxn * dxn + dyn * dyn, df2 = dxf * dxf + dyf * dyf;
    if (dn2 > r_out2) return;
    // cells of the row that meet the outer ball
    const float zr = sqrtf(r_out2 - dn2);
    // (index arithmetic in float32 carries 1e-3 of a cell width of slack,
    // far above its rounding for G <= 1024)
    const float gz = (float)G;
    const int zlo = (int)floorf(fminf(fmaxf((q.z - zr - m - g.lo[2]) * g.scale[2] - 1e-3f, -2.0f), gz + 1.0f));
    const int zhi = (int)floorf(fminf(fmaxf((q.z + zr + m - g.lo[2]) * g.scale[2] + 1e-3f, -2.0f), gz + 1.0f));
    // cells of the row wholly inside the inner ball: [zi0, zi1]
    int zi0 = 1, zi1 = 0;
    if (r_in2 > df2) {
        const float zi = sqrtf(r_in2 - df2);
        zi0 = (int)ceilf(fminf(fmaxf((q.z - zi + m - g.lo[2]) * g.scale[2] + 1e-3f, -2.0f), gz + 1.0f));
        zi1 = (int)floorf(fminf(fmaxf((q.z + zi - m - g.lo[2]) * g.scale[2] - 1e-3f, -2.0f), gz + 1.0f)) - 1;
    }
    const bool rim = dx == -s || dx == s || dy == -s || dy == s;
    const int base = (x * G + y) * G;
    int za, zb;
    if (rim) {
        za = iz - s > zlo ? iz - s : zlo;
        zb = iz + s < zhi ? iz + s : zhi;
        za = za < 0 ? 0 : za;
        zb = zb > G - 1 ? G - 1 : zb;
        if (za > zb) return;
        if (zi0 <= zi1 && zi0 <= zb && zi1 >= za) {  // the inner cells split the run
            if (half) za = zi1 + 1 > za ? zi1 + 1 : za;
            else zb = zi0 - 1 < zb ? zi0 - 1 : zb;
        } else if (half) {
            return;
        }
    } else {
        const int z = half ? iz + s : iz - s;
        if (z < 0 || z >= G || z < zlo || z > zhi || (z >= zi0 && z <= zi1)) return;
        za = zb = z;
    }
    if (za > zb) return;
    a = cell_off[base + za];
    b = cell_off[base + zb + 1];
}

// ---------------------------------------------------------------------------
// periodic boxes: candidates are images p_j + t L, t in [-2, 2]^3. A list
// entry (or plane source) packs the sorted index j in bits 0..23 with the
// image code (tx+2)*25 + (ty+2)*5 + (tz+2) in bits 24..30; IMG_NONE (62) is
// t = 0. Ties between equal keys go by (original index, code): the tie key
// orig * 128 + code. Outside periodic boxes entries are plain indices.
// ---------------------------------------------------------------------------
constexpr int IMG_NONE = 62;
constexpr int32_t IMG_INDEX_MASK = (1 << 24) - 1;

__device__ __forceinline__ int img_code(int tx, int ty, int tz) { return (tx + 2) * 25 + (ty + 2) * 5 + (tz + 2); }
__device__ __forceinline__ void img_t(int code, int& tx, int& ty, int& tz)
{
    tx = code / 25 - 2;
    ty = (code / 5) % 5 - 2;
    tz = code % 5 - 2;
}
__device__ __forceinline__ int img_pack(int j, int code) { return j | (code << 24); }
__device__ __forceinline__ int img_index(int jp, const GridDesc& g) { return g.periodic ? (jp & IMG_INDEX_MASK) : jp; }
__device__ __forceinline__ int img_code_of(int jp, const GridDesc& g)
{
    return g.periodic ? (int)((unsigned)jp >> 24) : IMG_NONE;
}
// tie key of a candidate: its original index, times 128 plus its code when periodic
__device__ __forceinline__ int img_tie(float4 pc, int code, const GridDesc& g)
{
    return g.periodic ? __float_as_int(pc.w) * 128 + code : __float_as_int(pc.w);
}
// one coordinate of the offset p_j + t L - p_i in float32: a shifted
// coordinate is formed in double and rounded once (forming c + t L in
// float32 first would lose up to an ulp of the period, far more than the
// offset of a close neighbour across the boundary can bear)
__device__ __forceinline__ float img_d(float c, float q, int t, float lo, float hi)
{
    return t == 0 ? c - q : (float)(((double)c - (double)q) + (double)t * ((double)hi - (double)lo));
}
// the same in double, every operation separately rounded: the exact key's
// coordinate (t = 0 adds nothing: x + 0 = x, and the FP64 pipe is scarce)
__device__ __forceinline__ double img_d64(float c, float q, int t, float lo, float hi)
{
    const double d = __dsub_rn((double)c, (double)q);
    return t == 0 ? d : __dadd_rn(d, (double)t * __dsub_rn((double)hi, (double)lo));
}
// compile-time forms for kernels instantiated per box kind (PER = periodic)
template <bool PER>
__device__ __forceinline__ int img_index_t(int jp) { return PER ? (jp & IMG_INDEX_MASK) : jp; }
template <bool PER>
__device__ __forceinline__ int img_code_t(int jp) { return PER ? (int)((unsigned)jp >> 24) : IMG_NONE; }
template <bool PER>
__device__ __forceinline__ int img_tie_t(float4 pc, int code)
{
    return PER ? __float_as_int(pc.w) * 128 + code : __float_as_int(pc.w);
}

// float32 offset of candidate pc (code) from pq
__device__ __forceinline__ float3 img_off(float4 pq, float4 pc, int code, const GridDesc& g)
{
    if (code == IMG_NONE) return make_float3(pc.x - pq.x, pc.y - pq.y, pc.z - pq.z);
    int tx, ty, tz;
    img_t(code, tx, ty, tz);
    return make_float3(img_d(pc.x, pq.x, tx, g.lo[0], g.hi[0]), img_d(pc.y, pq.y, ty, g.lo[1], g.hi[1]),
                       img_d(pc.z, pq.z, tz, g.lo[2], g.hi[2]));
}

// kNN ordering keys. FP64 form: ((dx*dx + dy*dy) + dz*dz) in double with
// dx = double(x_j) - double(x_i), every operation separately rounded (no FMA),
// so lists are exact and reproducible. FP32 form: the same in float32 with FMA.
__device__ __forceinline__ double knn_d2_f64(float4 a, float4 b)
{
    const double dx = __dsub_rn((double)b.x, (double)a.x);
    const double dy = __dsub_rn((double)b.y, (double)a.y);
    const double dz = __dsub_rn((double)b.z, (double)a.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
__device__ __forceinline__ float knn_d2_f32(float4 a, float4 b)
{
    const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}
__device__ __forceinline__ float key_f32(float3 o) { return fmaf(o.z, o.z, fmaf(o.y, o.y, o.x * o.x)); }
template <bool PER>
__device__ __forceinline__ float3 img_off_t(float4 pq, float4 pc, int code, const GridDesc& g)
{
    if (!PER) return make_float3(pc.x - pq.x, pc.y - pq.y, pc.z - pq.z);
    return img_off(pq, pc, code, g);
}

// the FP64 key of packed candidate jp (periodic: its image) from pq
__device__ __forceinline__ double img_key64(float4 pq, const float4* __restrict__ sorted, int jp, const GridDesc& g)
{
    if (!g.periodic || (int)((unsigned)jp >> 24) == IMG_NONE) return knn_d2_f64(pq, sorted[jp & (g.periodic ? IMG_INDEX_MASK : -1)]);
    const float4 pc = sorted[jp & IMG_INDEX_MASK];
    int tx, ty, tz;
    img_t((int)((unsigned)jp >> 24), tx, ty, tz);
    const double dx = img_d64(pc.x, pq.x, tx, g.lo[0], g.hi[0]);
    const double dy = img_d64(pc.y, pq.y, ty, g.lo[1], g.hi[1]);
    const double dz = img_d64(pc.z, pq.z, tz, g.lo[2], g.hi[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------
// periodic shell walk. Shell s of a periodic grid is walked in unwrapped grid
// coordinates; a cell (x, y, z) is the grid cell (x mod G, ...) seen through
// the image t = (floor(x / G), ...). A rim row's z-run crosses image
// boundaries, so each row owns seg_per_row segments: pieces of one z-image
// each, every piece split in the part below and above the inner ball.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ int seg_per_row(const GridDesc& g, int s)
{
    if (!g.periodic) return 2;
    const int W = 2 * s + 1;
    return 2 * (W <= g.G ? 2 : (W + g.G - 1) / g.G + 1);
}

// segments per row when no inner ball is skipped (the kNN): one per z-image piece
__device__ __forceinline__ int seg_per_row_outer(const GridDesc& g, int s)
{
    const int W = 2 * s + 1;
    return W <= g.G ? 2 : (W + g.G - 1) / g.G + 1;
}

// |L| of a periodic box: no image farther than this can cut a cell
__device__ __forceinline__ float period_norm2(const GridDesc& g)
{
    const float lx = g.hi[0] - g.lo[0], ly = g.hi[1] - g.lo[1], lz = g.hi[2] - g.lo[2];
    return lx * lx + ly * ly + lz * lz;
}

// distance from q to the outside of the block of shells 0..s (no walls), less
// the rounding margin
__device__ __forceinline__ float shell_gap_p(const GridDesc& g, float4 q, int ix, int iy, int iz, int s)
{
    const float c0 = (float)g.cw[0], c1 = (float)g.cw[1], c2 = (float)g.cw[2];
    float gap = fminf(q.x - (g.lo[0] + (float)(ix - s) * c0), (g.lo[0] + (float)(ix + s + 1) * c0) - q.x);
    gap = fminf(gap, fminf(q.y - (g.lo[1] + (float)(iy - s) * c1), (g.lo[1] + (float)(iy + s + 1) * c1) - q.y));
    gap = fminf(gap, fminf(q.z - (g.lo[2] + (float)(iz - s) * c2), (g.lo[2] + (float)(iz + s + 1) * c2) - q.z));
    return gap - 2.0f * (float)g.margin;
}

// Segment e (of M = seg_per_row per row) of periodic shell s, restricted to
// cells that reach into the ball r_out2 around q and are not wholly inside
// the ball r_in2 (see shell_segment_ball): the sorted range [a, b) and the
// image code of its cells. Images beyond t = +-2 are never returned (no
// generator there can cut a cell of a box with |L| <= 2 min L_a).
__device__ __forceinline__ void shell_segment_ball_p(int e, int s, int M, int ix, int iy, int iz, const GridDesc& g,
                                                     const int32_t* __restrict__ cell_off, float4 q, float r_out2,
                                                     float r_in2, int& a, int& b, int& code)
{
    const int G = g.G;
    const int W = 2 * s + 1;
    const int row = e / M, sub = e - (e / M) * M, piece = sub >> 1, half = sub & 1;
    const int dx = row / W - s, dy = row - (row / W) * W - s;
    const int x = ix + dx, y = iy + dy;
    a = b = 0;
    code = IMG_NONE;
    const int tx = floordiv(x, G), ty = floordiv(y, G);
    if (tx < -2 || tx > 2 || ty < -2 || ty > 2) return;
    const float m = (float)g.margin;
    const float cx = (float)g.cw[0], cy = (float)g.cw[1];
    const float x0 = g.lo[0] + (float)x * cx - m, x1 = g.lo[0] + (float)(x + 1) * cx + m;
    const float y0 = g.lo[1] + (float)y * cy - m, y1 = g.lo[1] + (float)(y + 1) * cy + m;
    const float dxn = fmaxf(fmaxf(x0 - q.x, q.x - x1), 0.0f), dyn = fmaxf(fmaxf(y0 - q.y, q.y - y1), 0.0f);
    const float dxf = fmaxf(q.x - x0, x1 - q.x), dyf = fmaxf(q.y - y0, y1 - q.y);
    const float dn2 = dxn * dxn + dyn * dyn, df2 = dxf * dxf + dyf * dyf;
    if (dn2 > r_out2) return;
    const float zr = sqrtf(r_out2 - dn2);
    const float zmax = 8.0f * (float)G;  // far beyond any image t in [-2, 2]
    const int zlo = (int)floorf(fminf(fmaxf((q.z - zr - m - g.lo[2]) * g.scale[2] - 1e-3f, -zmax), zmax));
    const int zhi = (int)floorf(fminf(fmaxf((q.z + zr + m - g.lo[2]) * g.scale[2] + 1e-3f, -zmax), zmax));
    int zi0 = 1, zi1 = 0;
    if (r_in2 > df2) {
        const float zi = sqrtf(r_in2 - df2);
        zi0 = (int)ceilf(fminf(fmaxf((q.z - zi + m - g.lo[2]) * g.scale[2] + 1e-3f, -zmax), zmax));
        zi1 = (int)floorf(fminf(fmaxf((q.z + zi - m - g.lo[2]) * g.scale[2] - 1e-3f, -zmax), zmax)) - 1;
    }
    const bool rim = dx == -s || dx == s || dy == -s || dy == s;
    int za, zb, tz;
    if (rim) {
        tz = floordiv(iz - s, G) + piece;
        za = iz - s > zlo ? iz - s : zlo;
        zb = iz + s < zhi ? iz + s : zhi;
        za = za > tz * G ? za : tz * G;
        zb = zb < tz * G + G - 1 ? zb : tz * G + G - 1;
        if (za > zb) return;
        if (zi0 <= zi1 && zi0 <= zb && zi1 >= za) {  // the inner cells split this piece
            if (half) za = zi1 + 1 > za ? zi1 + 1 : za;
            else zb = zi0 - 1 < zb ? zi0 - 1 : zb;
        } else if (half) {
            return;
        }
    } else {
        if (piece != 0) return;
        const int z = half ? iz + s : iz - s;
        if (z < zlo || z > zhi || (z >= zi0 && z <= zi1)) return;
        za = zb = z;
        tz = floordiv(z, G);
    }
    if (za > zb || tz < -2 || tz > 2) return;
    const int base = ((x - tx * G) * G + (y - ty * G)) * G - tz * G;
    a = cell_off[base + za];
    b = cell_off[base + zb + 1];
    code = img_code(tx, ty, tz);
}

// The same without an inner ball (M = seg_per_row_outer segments per row):
// a rim row's segments are its z-image pieces, an inner row's are its two
// cells z = iz - s and z = iz + s.
__device__ __forceinline__ void shell_segment_outer_p(int e, int s, int M, int ix, int iy, int iz, const GridDesc& g,
                                                      const int32_t* __restrict__ cell_off, float4 q, float r_out2,
                                                      int& a, int& b, int& code)
{
    const int G = g.G;
    const int W = 2 * s + 1;
    const int row = e / M, piece = e - (e / M) * M;
    const int dx = row / W - s, dy = row - (row / W) * W - s;
    const int x = ix + dx, y = iy + dy;
    a = b = 0;
    code = IMG_NONE;
    const int tx = floordiv(x, G), ty = floordiv(y, G);
    if (tx < -2 || tx > 2 || ty < -2 || ty > 2) return;
    const float m = (float)g.margin;
    const float cx = (float)g.cw[0], cy = (float)g.cw[1];
    const float x0 = g.lo[0] + (float)x * cx - m, x1 = g.lo[0] + (float)(x + 1) * cx + m;
    const float y0 = g.lo[1] + (float)y * cy - m, y1 = g.lo[1] + (float)(y + 1) * cy + m;
    const float dxn = fmaxf(fmaxf(x0 - q.x, q.x - x1), 0.0f), dyn = fmaxf(fmaxf(y0 - q.y, q.y - y1), 0.0f);
    const float dn2 = dxn * dxn + dyn * dyn;
    if (dn2 > r_out2) return;
    const float zr = sqrtf(r_out2 - dn2);
    const float zmax = 8.0f * (float)G;
    const int zlo = (int)floorf(fminf(fmaxf((q.z - zr - m - g.lo[2]) * g.scale[2] - 1e-3f, -zmax), zmax));
    const int zhi = (int)floorf(fminf(fmaxf((q.z + zr + m - g.lo[2]) * g.scale[2] + 1e-3f, -zmax), zmax));
    const bool rim = dx == -s || dx == s || dy == -s || dy == s;
    int za, zb, tz;
    if (rim) {
        tz = floordiv(iz - s, G) + piece;
        za = iz - s > zlo ? iz - s : zlo;
        zb = iz + s < zhi ? iz + s : zhi;
        za = za > tz * G ? za : tz * G;
        zb = zb < tz * G + G - 1 ? zb : tz * G + G - 1;
    } else {
        if (piece > 1) return;
        const int z = piece ? iz + s : iz - s;
        if (z < zlo || z > zhi) return;
        za = zb = z;
        tz = floordiv(z, G);
    }
    if (za > zb || tz < -2 || tz > 2) return;
    const int base = ((x - tx * G) * G + (y - ty * G)) * G - tz * G;
    a = cell_off[base + za];
    b = cell_off[base + zb + 1];
    code = img_code(tx, ty, tz);
}

// ---------------------------------------------------------------------------
// header of a cell's saved polyhedron between passes (fixed stride per cell;
// the planes, topology and positions follow at 128 bytes)
// ---------------------------------------------------------------------------
struct StateHdr {
    uint64_t alive[2];
    int32_t np;
    int32_t last_orig;   // original index of the last list entry processed
    double R2;           // max |v|^2 over the vertices (local frame)
    double last_d2;      // the last list entry's kNN key
    float bb_lo[3];      // bounding box of the vertices (local frame)
    float bb_hi[3];
    int32_t pad[4];
};
static_assert(sizeof(StateHdr) <= 128, "state header");


// ---------------------------------------------------------------------------
// device status block at the start of every workspace
// ---------------------------------------------------------------------------
struct DevStatus {
    int32_t bad_point;        // 1 + smallest offending input index, 0 if none
    int32_t duplicate;        // nonzero once a neighbour at distance 0 was seen
    int32_t n_fail_next;      // cells that need the next k (failed validation)
    int32_t n_fail_robust;    // cells that need the robust variant (capacity / precision)
    int32_t n_big_cells;      // grid cells too large for the per-thread fix-up sort
    int32_t record_overflow;  // cells whose final polyhedron does not fit an output record
    int32_t cap_overflow;     // an output buffer was too small for the emitted data (device check)
    int32_t n_unval;          // cells left unvalidated (no-sync schedule)
    unsigned long long fp64_rechecks;
    unsigned long long capacity_events;
    unsigned long long precision_events;
    long long totals[4];      // nbr, vtx, face, face_vtx totals written by the emit scan
    unsigned int detail[8];   // clip events: 0 keep-none, 1 plane cap, 2 vertex cap, 3 ring, 4 interpolated
    int32_t n_second;         // cells of a merged first pass still open at entry k (stats)
    int32_t n_range_over;     // cells of the last pass with more candidates than a range list holds
    unsigned long long knn_evals;    // candidate distances the k-nearest-neighbour kernels evaluated
    unsigned long long knn_queries;  // queries they answered
    int32_t check_fail;       // VT_CHECKS builds: code of the first failed bounds check, else 0
    int32_t pad0;
    unsigned long long walk_cells;  // last-pass walks over the shells within 2R (range lists, clipper)
    unsigned long long walk_cands;  // generators of the grid runs those walks examined
    int32_t pad[6];
};
static_assert(sizeof(DevStatus) % 64 == 0, "status block must stay 64-byte sized");

// Debug builds (-DVT_CHECKS): every shared-memory plane or vertex-slot index
// that comes from data (topology links, list entries) and every output-record
// and CSR index is checked against its bound; a bad one records its code in
// the status block (the call then returns VT_ERR_INTERNAL) and is replaced
// by 0, so the access stays in bounds. Without the flag the checks compile
// to nothing.
#ifdef VT_CHECKS
constexpr bool VT_CHECKED = true;
#else
constexpr bool VT_CHECKED = false;
#endif
enum { CK_PLANE = 1, CK_SLOT = 2, CK_EDGE = 3, CK_RECORD = 4, CK_CSR = 5 };
__device__ __forceinline__ int vt_ck(int i, int cap, int code, DevStatus* st)
{
    if (VT_CHECKED && (unsigned)i >= (unsigned)cap) {
        atomicCAS(&st->check_fail, 0, code);
        return 0;
    }
    return i;
}

// candidate lists of the last pass (range.cu): at most RANGE_CAP per cell
// (64 measured as fast as 96 and faster than 128 on the 1M mixed cloud)
#ifndef VT_RANGE_CAP
#define VT_RANGE_CAP 64
#endif
constexpr int RANGE_CAP = VT_RANGE_CAP;
struct RangeArgs {
    const float4* sorted;
    const int32_t* cell_off;
    GridDesc g;
    const GridDesc* sets;
    const int32_t* set_of;
    const int32_t* queries;  // sorted indices of the cells (saved states), from entry nq_off
    int64_t nq;              // cells (the bound when nq_dev is set)
    const int32_t* nq_dev;
    int64_t nq_off;
    const uint8_t* state;
    size_t state_stride;
    size_t pos_off;          // offset of the saved vertex positions (Real[3][64]) in a state
    int precision;           // key and position precision: VT_FP64 or VT_FP32_RECHECK
    int32_t* rnbr;           // [nq * RANGE_CAP] sorted indices, nearest first
    void* rd2;               // [nq * RANGE_CAP] their keys (float or double)
    int32_t* rlen;           // [nq] list length, -1 when the cell overflowed
    int32_t* over_list;      // overflowed cells (appended)
    int32_t* over_ctr;
    DevStatus* st;
    int32_t* queue;          // the launch's cell counter (zeroed by the launch)
};
cudaError_t launch_range(const RangeArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// per-cell output record (fixed stride, in the workspace)
// ---------------------------------------------------------------------------
constexpr int REC_FACES = 64;      // faces of a final cell
constexpr int REC_VERTS = 128;     // vertices of a final cell
struct RecHeader {
    int32_t nnbr;                  // neighbours kept (area > threshold)
    int32_t nface;                 // faces written (geometry)
    int32_t nvtx;                  // vertices written (geometry)
    int32_t nfv;                   // face-vertex entries (geometry)
    float p[3];                    // the generator (float32 vertex records hold offsets from it)
    int32_t pad;
};
// layout: RecHeader | int32 nbr[REC_FACES] | (geometry:) int32 face_nbr[REC_FACES] |
//         uint8 face_deg[REC_FACES] | uint8 face_vtx[3*REC_VERTS] | vtx[REC_VERTS*3]:
// in the FP32 form float offsets from the generator (emit adds them to it in
// FP64: the same values as adding the float vertex to the float generator in
// FP64), in the FP64 form FP64 coordinates
constexpr size_t REC_NBR_OFF = sizeof(RecHeader);
constexpr size_t REC_FNBR_OFF = REC_NBR_OFF + 4 * REC_FACES;
constexpr size_t REC_FDEG_OFF = REC_FNBR_OFF + 4 * REC_FACES;
constexpr size_t REC_FVTX_OFF = REC_FDEG_OFF + REC_FACES;
constexpr size_t REC_VTX_OFF = (REC_FVTX_OFF + 3 * REC_VERTS + 15) / 16 * 16;
constexpr size_t REC_STRIDE_NBR = REC_FNBR_OFF;                              // 288 B
constexpr size_t REC_STRIDE_GEOM_F32 = REC_VTX_OFF + 4 * 3 * REC_VERTS;      // ~2.6 KB
constexpr size_t REC_STRIDE_GEOM = REC_VTX_OFF + 8 * 3 * REC_VERTS;          // ~4.1 KB

// fail reasons stored per cell
enum : int8_t { CELL_DONE = 0, CELL_NEED_K = 1, CELL_NEED_ROBUST = 2, CELL_UNVALIDATED = 3 };

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
// the cell counter of a clip launch, in the workspace's counter region
constexpr int CTR_QUEUE = 4 * VT_MAX_PASSES + 4;

struct Layout {
    int G;
    int64_t n, g3;
    int64_t knn_cap;            // entries of the neighbour-list buffer
    int64_t rob_cap;            // entries of the robust variant's list buffer
    size_t rec_stride;
    size_t status, cid, ticket, counts, cell_off, big, scan_tmp, sorted, perm;
    size_t state_stride;
    size_t list_a, list_b, list_r, knn_nbr, knn_d2, rob_nbr, rob_d2, rec, cnt, off64, scan_emit, state, set_of, ctr,
        rlen;
    size_t total;
};
// cells < 0: the single-set grid of p; otherwise the total grid cells of a batch
Layout make_layout(const vt_params* p, int64_t n, int64_t cells = -1, bool batch = false);

// ---------------------------------------------------------------------------
// launch helpers shared by the translation units
// ---------------------------------------------------------------------------
int set_error(int code, const char* msg);  // records msg for vt_last_error, returns code
// VT_ERR_INVALID_ARG (naming the buffer) unless every non-NULL ptrs[i] is
// memory device code can use (device, managed or pinned host); skipped while
// `stream` is being captured
int check_device_buffers(void* stream, const void* const* ptrs, const char* const* names, int count);
void count_launch(int n = 1);
int64_t launches();

// exclusive scans (grid-wide, multi-kernel); tmp needs scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s);
void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s);

// stage launchers (return cudaError_t of the launch)
// batches: sets (device, nsets descriptors), set_off (device, nsets + 1 point
// offsets), g3 = total grid cells of all sets; set_of receives the set of each
// sorted point. A single set passes sets = set_off = set_of = nullptr.
struct BatchArgs {
    const GridDesc* sets;
    const int64_t* set_off;
    int nsets;
    int32_t* set_of;
};
cudaError_t launch_grid_build(const float* pts, int64_t n, const GridDesc& g, float4* sorted, int32_t* perm,
                              int32_t* cell_off, int32_t* cid, int32_t* ticket, int32_t* counts, int32_t* big,
                              void* scan_tmp, DevStatus* st, cudaStream_t s, const BatchArgs* batch = nullptr,
                              int64_t g3 = -1);

// acc[s] = sum over the grid cells of set s of n_c (n_c - 1) (sets = nullptr: one set)
cudaError_t launch_pair_counts(const int32_t* cell_off, int64_t g3, const GridDesc* sets, int nsets,
                               unsigned long long* acc, cudaStream_t s);

// nq_dev: the query count is read from device memory; the launch takes list
// entries [nq_off, nq_off + nq) (queries already points at entry nq_off)
cudaError_t launch_knn(const float4* sorted, const int32_t* cell_off, const GridDesc& g, int64_t n,
                       const int32_t* queries, int64_t nq, int k, int precision, int32_t* nbr, void* d2,
                       DevStatus* st, cudaStream_t s, const GridDesc* sets = nullptr, const int32_t* set_of = nullptr,
                       const int32_t* nq_dev = nullptr, int64_t nq_off = 0, int32_t* queue = nullptr);

struct ClipArgs {
    const float4* sorted;
    const int32_t* cell_off;
    GridDesc g;
    int64_t n;
    const int32_t* queries;   // sorted indices (NULL = 0..nq-1)
    int64_t nq;
    const int32_t* nbr;       // [nq*k] (k > 0)
    const void* d2;           // [nq*k] float or double
    int k;                    // list entries per cell (0 = no list; the stride of nbr/d2)
    int exhaustive;           // 1: after the list (or the resumed state), walk every generator within 2R
    const int32_t* klen;      // per-cell list lengths (<= k), or NULL (every list has k entries)
    int kstride;              // entries per cell in nbr / d2 (0: k)
    int k_next;               // > k: a cell the first k entries leave open continues with
                              // entries [k, k_next) in the same launch (the doubled list)
    int by_cell;              // 1: lists are indexed by the cell's sorted index, not its position
    int complete;             // 1: the lists hold every generator that can still cut (range lists)
    int restore;              // 1: resume the saved state and start at list entry 0
    int emit;
    int index_space;
    double* vol;
    double* cen;
    double* m2;
    uint8_t* rec;             // records base (NULL = none)
    size_t rec_stride;
    int32_t* fail_next;       // appended: cells needing a larger k
    int32_t* fail_robust;     // appended: cells needing the robust variant (or, from
                              // the robust variant itself, cells left unvalidated)
    int32_t* ctr_next;        // device counters of the two lists
    int32_t* ctr_robust;
    const GridDesc* sets;     // per-set grids of a batch (NULL: the single grid g)
    const int32_t* set_of;    // set of each sorted point (batches)
    const int32_t* nq_dev;    // when set, the cell count is read from device memory
    int64_t nq_cap;           // with nq_dev: at most this many cells per launch (the list buffers)
    int64_t nq_off;           // with nq_dev: this launch takes list entries [nq_off, nq_off + nq_cap)
    int k_prev;               // > 0: resume saved cells; list entries [0, k_prev) are done
    uint8_t* state;           // per-cell saved polyhedra (sorted index * state_stride), or NULL
    size_t state_stride;
    DevStatus* st;
    int32_t* queue;           // the launch's cell counter (zeroed by the launch)
    int rec_f32;              // geometry records hold float offsets from the generator (the FP32 form)
};
// variant: 0 = FP32 regular, 1 = FP64 regular, 2 = FP64 robust (bigger capacity),
// 3 = FP32 with the robust capacity (the FP32 form's first fallback)
cudaError_t launch_clip(const ClipArgs& a, int variant, int threads_per_cell, cudaStream_t s);
size_t clip_state_bytes(int precision);       // per-cell state of the regular variant (64 slots)
size_t clip_state_pos_offset(int precision);  // offset of its vertex positions: Real[3][64], x, y, z rows

struct EmitArgs {
    int64_t n;
    int emit;
    int vtx_f32;              // vertex records: float offsets from the generator (see RecHeader)
    const uint8_t* rec;
    size_t rec_stride;
    int32_t* cnt;             // [4*n] scratch counts
    int64_t* off64;           // [4*(n+1)] scratch offsets
    void* scan_tmp;
    DevStatus* st;
};
cudaError_t launch_emit_count(const EmitArgs& a, cudaStream_t s);  // counts + scans + totals
cudaError_t launch_emit_write(const EmitArgs& a, const vt_cells_out& out, cudaStream_t s);  // device-checked caps
// NaN into vol / cen / m2 of the unvalidated cells list[count] (count = *n_dev
// when set, else n_host; n_bound sizes the grid)
cudaError_t launch_mark_unvalidated(const int32_t* list, const int32_t* n_dev, int64_t n_host, int64_t n_bound,
                                    const float4* sorted, int index_space, double* vol, double* cen, double* m2,
                                    DevStatus* st, cudaStream_t s);
cudaError_t launch_unvalidated_ids(const int32_t* list, int64_t cnt, const float4* sorted, int index_space,
                                   int32_t* ids, cudaStream_t s);
// Lloyd's update p <- p - grad / (2 vol), wrapped into a periodic box
cudaError_t launch_lloyd_step(const float* pts, int64_t n, const double* grad, const double* vol, const GridDesc& g,
                              float* out, cudaStream_t s);
// g: the box (lo, hi) and its periodic flag
cudaError_t launch_adjoint(const float* pts, int64_t n, const vt_cells_out& c, const double* gV, const double* gC,
                           const double* gM, double* grad, int precision, const GridDesc& g, cudaStream_t s);

}  // namespace vt
