// clip_impl.cuh -- stage 3: per-cell bisector clipping with the security-radius
// stop (votess paper, Summary: each cell is obtained by clipping a bounding
// box with the perpendicular bisectors between the generator and its nearest
// neighbours; a security-radius condition validates the cell).
//
// Work decomposition: T lanes (a "group", T = 8, 16 or 32, all inside one
// warp) build one cell at a time; groups stride over the cells.
//
// Representation of the convex polyhedron (local frame of the generator, so
// the generator is the origin):
//  * planes  n.x <= b in shared memory (SoA), with the source of each plane
//    (sorted index of the neighbour, or -1..-6 for the walls x-,x+,y-,y+,z-,z+);
//  * vertices in VCAP slots. Slot s lives in lane s % T, register row s / T
//    (positions in registers, so the per-plane sign pass touches no memory).
//    In shared memory each slot holds the three planes meeting at the vertex,
//    (a, b, c), ordered counter-clockwise seen from outside, and three
//    adjacency links: the vertex across the polyhedron edge between faces
//    a&b, b&c and c&a. A 128-bit mask marks the live slots.
//
// Clipping by a plane h: every lane tests its live vertices; removed vertices
// form a connected patch. Each edge (x -> y) of a removed vertex whose
// neighbour w across it survives is a boundary edge and yields one new vertex
// with planes (x, y, h) on the cut edge; its link across x&y is w, and the new
// vertices chain around h through start_of[x] / end_of[y] tables (each face
// x is cut at most once, so x starts exactly one boundary edge). New slots
// take the lowest free slots; their positions are solved from the three
// planes by the owning lanes.
//
// FP32 form (variant 0): planes, vertices and sign tests in float32. A sign
// test with |s| < 1e-6 |n| R is re-decided in FP64 from the vertex's three
// planes rebuilt in FP64 from the input points; the security-radius test is
// re-decided in FP64 (vertices re-solved in FP64) when it is within 1e-5
// relative of equality; volumes and moments accumulate per lane in float32 and
// across lanes in FP64. A topology inconsistency (a face cut twice, a singular
// vertex) sends the cell to the robust FP64 variant.
#pragma once
#include <float.h>
#include <limits.h>

#include "vt_internal.cuh"

namespace vt {

namespace {

// ---------------------------------------------------------------------------
// 128-bit slot mask
// ---------------------------------------------------------------------------
struct Mask {
    uint64_t w[2];
    __device__ __forceinline__ bool test(int s) const { return (w[s >> 6] >> (s & 63)) & 1ull; }
    __device__ __forceinline__ void set(int s) { w[s >> 6] |= 1ull << (s & 63); }
    __device__ __forceinline__ bool none() const { return (w[0] | w[1]) == 0; }
    __device__ __forceinline__ int count() const { return __popcll(w[0]) + __popcll(w[1]); }
    // number of set bits strictly below s
    __device__ __forceinline__ int rank(int s) const
    {
        if (s < 64) return __popcll(w[0] & ((1ull << s) - 1ull));
        return __popcll(w[0]) + __popcll(w[1] & ((1ull << (s - 64)) - 1ull));
    }
};

__device__ __forceinline__ Mask mask_and(Mask a, Mask b) { return {{a.w[0] & b.w[0], a.w[1] & b.w[1]}}; }
__device__ __forceinline__ Mask mask_or(Mask a, Mask b) { return {{a.w[0] | b.w[0], a.w[1] | b.w[1]}}; }
__device__ __forceinline__ Mask mask_not(Mask a, int cap)
{
    Mask m = {{~a.w[0], ~a.w[1]}};
    if (cap < 128) m.w[1] &= cap > 64 ? ((1ull << (cap - 64)) - 1ull) : 0ull;
    if (cap < 64) m.w[0] &= (1ull << cap) - 1ull;
    return m;
}
// position of the i-th (0-based) set bit, or -1
__device__ __forceinline__ int nth_set(Mask m, int i)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t lo = (uint32_t)m.w[h], hi = (uint32_t)(m.w[h] >> 32);
        int cl = __popc(lo);
        if (i < cl) return h * 64 + (int)__fns(lo, 0, i + 1);
        i -= cl;
        int ch = __popc(hi);
        if (i < ch) return h * 64 + 32 + (int)__fns(hi, 0, i + 1);
        i -= ch;
    }
    return -1;
}
// the first n set bits of m
__device__ __forceinline__ Mask first_n(Mask m, int n)
{
    if (n <= 0) return {{0ull, 0ull}};
    int last = nth_set(m, n - 1);
    Mask r = m;
    if (last < 64) {
        r.w[0] &= last == 63 ? ~0ull : ((1ull << (last + 1)) - 1ull);
        r.w[1] = 0;
    } else {
        int l = last - 64;
        r.w[1] &= l == 63 ? ~0ull : ((1ull << (l + 1)) - 1ull);
    }
    return r;
}

// ---------------------------------------------------------------------------
// group (T lanes of one warp) primitives
// ---------------------------------------------------------------------------
template <int T>
struct Group {
    unsigned mask;  // lanes of this group within the warp
    int base;       // first warp lane of the group
    int gl;         // lane within the group
    __device__ __forceinline__ Group()
    {
        const int wl = threadIdx.x & 31;
        base = (wl / T) * T;
        gl = wl - base;
        mask = T == 32 ? 0xffffffffu : (((1u << T) - 1u) << base);
    }
    __device__ __forceinline__ unsigned ballot(bool p) const
    {
        unsigned b = __ballot_sync(mask, p);
        return T == 32 ? b : (b >> base) & ((1u << T) - 1u);
    }
    __device__ __forceinline__ bool any(bool p) const { return ballot(p) != 0; }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    template <typename V>
    __device__ __forceinline__ V bcast(V v, int src) const { return __shfl_sync(mask, v, src, T); }
    template <typename V>
    __device__ __forceinline__ V max(V v) const
    {
#pragma unroll
        for (int o = T / 2; o >= 1; o >>= 1) { V u = __shfl_xor_sync(mask, v, o, T); v = u > v ? u : v; }
        return v;
    }
    template <typename V>
    __device__ __forceinline__ V sum(V v) const
    {
#pragma unroll
        for (int o = T / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(mask, v, o, T);
        return v;
    }
    __device__ __forceinline__ uint64_t orr(uint64_t v) const
    {
#pragma unroll
        for (int o = T / 2; o >= 1; o >>= 1) v |= __shfl_xor_sync(mask, v, o, T);
        return v;
    }
    // exclusive prefix sum and total
    __device__ __forceinline__ int scan(int v, int& total) const
    {
        int inc = v;
#pragma unroll
        for (int d = 1; d < T; d <<= 1) {
            int u = __shfl_up_sync(mask, inc, d, T);
            if (gl >= d) inc += u;
        }
        total = __shfl_sync(mask, inc, T - 1, T);
        return inc - v;
    }
};

// ---------------------------------------------------------------------------
// FP64 helpers (exact planes from the float32 inputs)
// ---------------------------------------------------------------------------
struct P64 { double x, y, z, b; };

__device__ __forceinline__ P64 plane64(int src, const float4* __restrict__ sorted, float4 pi, const GridDesc& g)
{
    P64 p;
    if (src >= 0) {
        float4 pj = sorted[src];
        p.x = (double)pj.x - (double)pi.x;
        p.y = (double)pj.y - (double)pi.y;
        p.z = (double)pj.z - (double)pi.z;
        p.b = 0.5 * ((p.x * p.x + p.y * p.y) + p.z * p.z);
    } else {
        const int w = -src - 1, axis = w >> 1, upper = w & 1;
        p.x = p.y = p.z = 0.0;
        const double pc = axis == 0 ? (double)pi.x : (axis == 1 ? (double)pi.y : (double)pi.z);
        const double v = upper ? 1.0 : -1.0;
        if (axis == 0) p.x = v; else if (axis == 1) p.y = v; else p.z = v;
        p.b = upper ? (double)g.hi[axis] - pc : pc - (double)g.lo[axis];
    }
    return p;
}

template <typename Real>
__device__ __forceinline__ bool solve3(Real ax, Real ay, Real az, Real ab, Real bx, Real by, Real bz, Real bb, Real cx,
                                       Real cy, Real cz, Real cb, Real& x, Real& y, Real& z, Real cond = (Real)0)
{
    // v = (ab (B x C) + bb (C x A) + cb (A x B)) / (A . (B x C))
    Real bcx = by * cz - bz * cy, bcy = bz * cx - bx * cz, bcz = bx * cy - by * cx;
    Real cax = cy * az - cz * ay, cay = cz * ax - cx * az, caz = cx * ay - cy * ax;
    Real abx = ay * bz - az * by, aby = az * bx - ax * bz, abz = ax * by - ay * bx;
    Real det = ax * bcx + ay * bcy + az * bcz;
    if (!(det != (Real)0) || !isfinite(det)) return false;
    if (cond > (Real)0) {
        const Real na = ax * ax + ay * ay + az * az, nb = bx * bx + by * by + bz * bz, nc = cx * cx + cy * cy + cz * cz;
        if (det * det < cond * cond * na * nb * nc) return false;
    }
    Real inv = (Real)1 / det;
    x = (ab * bcx + bb * cax + cb * abx) * inv;
    y = (ab * bcy + bb * cay + cb * aby) * inv;
    z = (ab * bcz + bb * caz + cb * abz) * inv;
    return isfinite(x) && isfinite(y) && isfinite(z);
}

__device__ __forceinline__ bool vertex64(const P64& A, const P64& B, const P64& C, double& x, double& y, double& z)
{
    return solve3<double>(A.x, A.y, A.z, A.b, B.x, B.y, B.z, B.b, C.x, C.y, C.z, C.b, x, y, z);
}

// ---------------------------------------------------------------------------
// shared memory of one group
// ---------------------------------------------------------------------------
template <typename Real, int VCAP, int PCAP>
struct GroupSmem {
    Real pnx[PCAP], pny[PCAP], pnz[PCAP], pb[PCAP];
    int32_t psrc[PCAP];
    uint8_t vid[VCAP][4];   // planes a, b, c (ccw from outside)
    uint8_t vadj[VCAP][4];  // neighbour across a&b, b&c, c&a
    uint8_t vsrc[VCAP];     // removed vertex whose cut edge created the slot (this clip)
    union {
        struct {
            uint32_t start_of[PCAP];  // (stamp << 8) | slot
            uint32_t end_of[PCAP];
        } ring;
        struct {
            Real area[PCAP];
            int32_t key[PCAP];
            int16_t first[PCAP];
            uint8_t deg[PCAP];
        } tail;
    } u;
    Real vpos[VCAP][3];
};

enum ClipResult { CLIP_NONE = 0, CLIP_CUT = 1, CLIP_OVERFLOW = 2, CLIP_INCONSISTENT = 3 };
enum CellEnd { END_VALID = 0, END_NEED_K = 1, END_OVERFLOW = 2, END_INCONSISTENT = 3 };

template <typename Real>
struct Tol;
// A vertex counts as outside a plane n.x <= b when s = n.v - b exceeds
// on_plane_rel * |n| * R (R = cell radius): round-off of FP64 vertex
// positions at exactly degenerate inputs (lattices) must not cut slivers.
// A 3x3 solve whose determinant is below cond_rel * |A||B||C| is replaced by
// interpolation along the cut edge.
template <>
struct Tol<float> {
    static constexpr bool fp32 = true;
    static constexpr double area_rel = 1e-11;
    static constexpr double cond_rel = 1e-3;
};
template <>
struct Tol<double> {
    static constexpr bool fp32 = false;
    static constexpr double area_rel = 1e-12;
    static constexpr double cond_rel = 1e-9;
};
constexpr double ON_PLANE_REL2 = 1e-28;  // (1e-14)^2

template <typename Real, int T, int VPL, int PCAP>
struct Cell {
    static constexpr int VCAP = T * VPL;
    using S = GroupSmem<Real, VCAP, PCAP>;

    const Group<T>& G;
    S& sm;
    const float4* __restrict__ sorted;
    const GridDesc& grid;
    DevStatus* st;
    float4 pi;
    Real vx[VPL], vy[VPL], vz[VPL];
    Mask alive;
    int np;           // planes in use (ids < np)
    uint32_t stamp;   // clip counter for the ring tables (keeps counting across cells)
    Real R2;          // max |v|^2 over live vertices

    __device__ Cell(const Group<T>& g_, S& sm_, const float4* s_, const GridDesc& gd, DevStatus* st_)
        : G(g_), sm(sm_), sorted(s_), grid(gd), st(st_)
    {
    }

    __device__ __forceinline__ void update_r2()
    {
        Real m = 0;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            Real d = vx[r] * vx[r] + vy[r] * vy[r] + vz[r] * vz[r];
            if (alive.test(s) && d > m) m = d;
        }
        R2 = G.max(m);
    }

    // the box [lo, hi) in the frame of pi: walls 0..5, corners in slots 0..7
    __device__ void init_box()
    {
        const Real px = (Real)pi.x, py = (Real)pi.y, pz = (Real)pi.z;
        const Real lo[3] = {(Real)grid.lo[0] - px, (Real)grid.lo[1] - py, (Real)grid.lo[2] - pz};
        const Real hi[3] = {(Real)grid.hi[0] - px, (Real)grid.hi[1] - py, (Real)grid.hi[2] - pz};
        if (G.gl < 6) {
            const int w = G.gl, axis = w >> 1, upper = w & 1;
            sm.pnx[w] = axis == 0 ? (upper ? (Real)1 : (Real)-1) : (Real)0;
            sm.pny[w] = axis == 1 ? (upper ? (Real)1 : (Real)-1) : (Real)0;
            sm.pnz[w] = axis == 2 ? (upper ? (Real)1 : (Real)-1) : (Real)0;
            sm.pb[w] = upper ? hi[axis] : -lo[axis];
            sm.psrc[w] = -(w + 1);
        }
        if (G.gl < 8) {
            const int c = G.gl, sx = (c >> 2) & 1, sy = (c >> 1) & 1, sz = c & 1;
            int P[3] = {sx, 2 + sy, 4 + sz};
            const int nlo = (1 - sx) + (1 - sy) + (1 - sz);
            if (nlo & 1) { int t = P[1]; P[1] = P[2]; P[2] = t; }
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                sm.vid[c][e] = (uint8_t)P[e];
                // neighbour across P[e] & P[e+1]: flip the axis of the third plane
                const int axis = P[(e + 2) % 3] >> 1;
                sm.vadj[c][e] = (uint8_t)(c ^ (4 >> axis));
            }
            sm.vid[c][3] = 0;
            sm.vadj[c][3] = 0;
        }
        alive.w[0] = 0xffull;
        alive.w[1] = 0;
        np = 6;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (s < 8) {
                vx[r] = ((s >> 2) & 1) ? hi[0] : lo[0];
                vy[r] = ((s >> 1) & 1) ? hi[1] : lo[1];
                vz[r] = (s & 1) ? hi[2] : lo[2];
            } else {
                vx[r] = vy[r] = vz[r] = 0;
            }
        }
        G.sync();
        update_r2();
    }

    // FP64 re-decision of a sign test: vertex re-solved from its planes
    __device__ bool outside64(int s, const P64& h, int r)
    {
        uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
        P64 A = plane64(sm.psrc[ids & 0xff], sorted, pi, grid);
        P64 B = plane64(sm.psrc[(ids >> 8) & 0xff], sorted, pi, grid);
        P64 C = plane64(sm.psrc[(ids >> 16) & 0xff], sorted, pi, grid);
        double x, y, z;
        if (!vertex64(A, B, C, x, y, z)) { x = vx[r]; y = vy[r]; z = vz[r]; }
        const double sv = (h.x * x + h.y * y) + h.z * z - h.b;
        return sv > 0.0 && sv * sv > ON_PLANE_REL2 * 2.0 * h.b * (double)R2;
    }

    // FP64 security radius: vertices re-solved in FP64
    __device__ double r2_64()
    {
        double m = 0;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (alive.test(s)) {
                uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
                P64 A = plane64(sm.psrc[ids & 0xff], sorted, pi, grid);
                P64 B = plane64(sm.psrc[(ids >> 8) & 0xff], sorted, pi, grid);
                P64 C = plane64(sm.psrc[(ids >> 16) & 0xff], sorted, pi, grid);
                double x, y, z;
                if (vertex64(A, B, C, x, y, z)) {
                    double d = (x * x + y * y) + z * z;
                    m = d > m ? d : m;
                } else {
                    double d = (double)vx[r] * vx[r] + (double)vy[r] * vy[r] + (double)vz[r] * vz[r];
                    m = d > m ? d : m;
                }
            }
        }
        return G.max(m);
    }

    // true when no generator at squared distance >= dj can cut the cell
    __device__ bool radius_ok(Real dj, int jsrc)
    {
        if (!Tol<Real>::fp32) return (Real)4 * R2 <= dj;
        const float lhs = 4.0f * (float)R2, rhs = (float)dj;
        if (lhs <= rhs * (1.0f - 1e-5f)) return true;
        if (lhs > rhs * (1.0f + 1e-5f)) return false;
        if (G.gl == 0) atomicAdd(&st->fp64_rechecks, 1ull);
        double d64 = 1e300;
        if (jsrc >= 0) {
            P64 h = plane64(jsrc, sorted, pi, grid);
            d64 = 4.0 * h.b * 0.5;  // |n|^2 = 2b
        } else {
            d64 = (double)dj;
        }
        return 4.0 * r2_64() <= d64;
    }

    // clip by n.x <= b (plane source src)
    __device__ int clip(Real nx, Real ny, Real nz, Real b, int src)
    {
        Mask out = {{0ull, 0ull}};
        bool near = false;
        Real sv[VPL];
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            sv[r] = nx * vx[r] + ny * vy[r] + nz * vz[r] - b;
            const bool al = alive.test(s);
            const bool o = al && sv[r] > (Real)0 &&
                           (Tol<Real>::fp32 || (double)sv[r] * sv[r] > ON_PLANE_REL2 * 2.0 * (double)b * (double)R2);
            if (Tol<Real>::fp32 && al && (float)sv[r] * (float)sv[r] < 2e-12f * (float)b * (float)R2) near = true;
            const uint64_t bits = G.ballot(o);
            const int sh = r * T;
            out.w[sh >> 6] |= bits << (sh & 63);
        }
        if (Tol<Real>::fp32 && G.any(near)) {
            // re-decide the near-zero tests in FP64
            P64 h = plane64(src, sorted, pi, grid);
            out.w[0] = out.w[1] = 0;
#pragma unroll
            for (int r = 0; r < VPL; ++r) {
                const int s = r * T + G.gl;
                const bool al = alive.test(s);
                bool o = al && sv[r] > (Real)0;
                if (al && (float)sv[r] * (float)sv[r] < 2e-12f * (float)b * (float)R2) {
                    o = outside64(s, h, r);
                    atomicAdd(&st->fp64_rechecks, 1ull);
                }
                const uint64_t bits = G.ballot(o);
                const int sh = r * T;
                out.w[sh >> 6] |= bits << (sh & 63);
            }
        }
        if (out.none()) return CLIP_NONE;
        const Mask keep = mask_and(alive, mask_not(out, 128));
        if (keep.none()) {  // the generator itself is always inside
            if (G.gl == 0) atomicAdd(&st->detail[0], 1u);
            return CLIP_INCONSISTENT;
        }

        // plane id for h
        int h = np;
        if (np >= PCAP) {
            uint64_t ref0 = 0, ref1 = 0;
#pragma unroll
            for (int r = 0; r < VPL; ++r) {
                const int s = r * T + G.gl;
                if (keep.test(s)) {
                    uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const int pid = (ids >> (8 * e)) & 0xff;
                        if (pid < 64) ref0 |= 1ull << pid; else ref1 |= 1ull << (pid - 64);
                    }
                }
            }
            ref0 = G.orr(ref0);
            ref1 = G.orr(ref1);
            Mask fr = mask_not(Mask{{ref0, ref1}}, PCAP);
            h = nth_set(fr, 0);
            if (h < 0) {
                if (G.gl == 0) atomicAdd(&st->detail[1], 1u);
                return CLIP_OVERFLOW;
            }
        }

        // boundary edges of the removed patch
        int mycnt = 0;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (out.test(s)) {
                uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[s]);
#pragma unroll
                for (int e = 0; e < 3; ++e) mycnt += out.test((adj >> (8 * e)) & 0xff) ? 0 : 1;
            }
        }
        int total;
        const int first = G.scan(mycnt, total);
        // new vertices go to slots that were free before this clip, so the
        // removed vertices' topology stays readable until the ring is closed
        const Mask freem = mask_not(alive, VCAP);
        if (total > freem.count()) {
            if (G.gl == 0) atomicAdd(&st->detail[2], 1u);
            return CLIP_OVERFLOW;
        }
        const Mask newm = first_n(freem, total);
        ++stamp;
        const uint32_t tag = stamp << 8;

        // new vertices: topology and ring tables
        int idx = first;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (out.test(s)) {
                const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
                const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[s]);
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const int w = (adj >> (8 * e)) & 0xff;
                    if (out.test(w)) continue;
                    const int d = nth_set(freem, idx++);
                    const int x = (ids >> (8 * e)) & 0xff, y = (ids >> (8 * ((e + 1) % 3))) & 0xff;
                    sm.vid[d][0] = (uint8_t)x;
                    sm.vid[d][1] = (uint8_t)y;
                    sm.vid[d][2] = (uint8_t)h;
                    sm.vid[d][3] = 0;
                    sm.vadj[d][0] = (uint8_t)w;
                    sm.vsrc[d] = (uint8_t)s;
                    sm.u.ring.start_of[x] = tag | (uint32_t)d;
                    sm.u.ring.end_of[y] = tag | (uint32_t)d;
                    // the survivor w: its link across y&x now points to d
                    const uint32_t wid = *reinterpret_cast<const uint32_t*>(sm.vid[w]);
#pragma unroll
                    for (int e2 = 0; e2 < 3; ++e2)
                        if ((int)((wid >> (8 * e2)) & 0xff) == y && (int)((wid >> (8 * ((e2 + 1) % 3))) & 0xff) == x)
                            sm.vadj[w][e2] = (uint8_t)d;
                }
            }
        }
        if (G.gl == 0) {
            sm.pnx[h] = nx;
            sm.pny[h] = ny;
            sm.pnz[h] = nz;
            sm.pb[h] = b;
            sm.psrc[h] = src;
        }
        G.sync();
        // close the ring around h
        bool bad = false;
        idx = first;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (out.test(s)) {
                const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
                const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[s]);
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const int w = (adj >> (8 * e)) & 0xff;
                    if (out.test(w)) continue;
                    const int d = nth_set(freem, idx++);
                    const int x = (ids >> (8 * e)) & 0xff, y = (ids >> (8 * ((e + 1) % 3))) & 0xff;
                    const uint32_t so = sm.u.ring.start_of[y], eo = sm.u.ring.end_of[x];
                    if ((so & ~0xffu) != tag || (eo & ~0xffu) != tag || sm.u.ring.start_of[x] != (tag | (uint32_t)d))
                        bad = true;
                    sm.vadj[d][1] = (uint8_t)(so & 0xff);
                    sm.vadj[d][2] = (uint8_t)(eo & 0xff);
                }
            }
        }
        if (G.any(bad)) {
            if (G.gl == 0) atomicAdd(&st->detail[3], 1u);
            return CLIP_INCONSISTENT;
        }
        if (h == np) ++np;
        alive = mask_or(keep, newm);
        G.sync();
        // positions of the new vertices, solved from their planes by the owners;
        // an ill-conditioned solve falls back to interpolation along the cut edge
        bool interp = false;
        uint32_t need = 0;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (newm.test(s)) {
                const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
                const int a = ids & 0xff, bb = (ids >> 8) & 0xff, c = (ids >> 16) & 0xff;
                if (!solve3<Real>(sm.pnx[a], sm.pny[a], sm.pnz[a], sm.pb[a], sm.pnx[bb], sm.pny[bb], sm.pnz[bb],
                                  sm.pb[bb], sm.pnx[c], sm.pny[c], sm.pnz[c], sm.pb[c], vx[r], vy[r], vz[r],
                                  (Real)Tol<Real>::cond_rel)) {
                    need |= 1u << r;
                    interp = true;
                }
            }
        }
        if (G.any(interp)) {
            if (G.gl == 0) atomicAdd(&st->detail[4], 1u);
            const Mask before = mask_or(keep, out);
#pragma unroll
            for (int r = 0; r < VPL; ++r) {
                const int s = r * T + G.gl;
                if (before.test(s)) {
                    sm.vpos[s][0] = vx[r];
                    sm.vpos[s][1] = vy[r];
                    sm.vpos[s][2] = vz[r];
                }
            }
            G.sync();
#pragma unroll
            for (int r = 0; r < VPL; ++r) {
                if (!((need >> r) & 1u)) continue;
                const int s = r * T + G.gl;
                const int v = sm.vsrc[s], w = sm.vadj[s][0];
                const Real px = sm.vpos[v][0], py = sm.vpos[v][1], pz = sm.vpos[v][2];
                const Real qx = sm.vpos[w][0], qy = sm.vpos[w][1], qz = sm.vpos[w][2];
                const Real sv_ = nx * px + ny * py + nz * pz - b, sw_ = nx * qx + ny * qy + nz * qz - b;
                Real t = sv_ - sw_ > (Real)0 ? sv_ / (sv_ - sw_) : (Real)0.5;
                t = t < (Real)0 ? (Real)0 : (t > (Real)1 ? (Real)1 : t);
                vx[r] = px + t * (qx - px);
                vy[r] = py + t * (qy - py);
                vz[r] = pz + t * (qz - pz);
            }
            G.sync();
        }
        update_r2();
        return CLIP_CUT;
    }

    __device__ __forceinline__ int clip_point(float4 pj, int j)
    {
        Real nx, ny, nz;
        if (Tol<Real>::fp32) {
            nx = (Real)(pj.x - pi.x);
            ny = (Real)(pj.y - pi.y);
            nz = (Real)(pj.z - pi.z);
        } else {
            nx = (Real)pj.x - (Real)pi.x;
            ny = (Real)pj.y - (Real)pi.y;
            nz = (Real)pj.z - (Real)pi.z;
        }
        const Real b = (Real)0.5 * (nx * nx + ny * ny + nz * nz);
        return clip(nx, ny, nz, b, j);
    }

    // ---------------------------------------------------------------------
    // moments, neighbours and geometry of a validated cell
    // ---------------------------------------------------------------------
    __device__ void finish(int64_t out_idx, const ClipArgs& A, int q)
    {
        // positions to shared memory, tables reset
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            sm.vpos[s][0] = vx[r];
            sm.vpos[s][1] = vy[r];
            sm.vpos[s][2] = vz[r];
        }
        for (int f = G.gl; f < np; f += T) {
            sm.u.tail.area[f] = 0;
            sm.u.tail.first[f] = -1;
        }
        G.sync();
        // per (vertex, face) terms: tetrahedron (0, q_f, v, next(v around f)),
        // q_f = foot of the perpendicular from the generator onto face f
        Real vol = 0, mx = 0, my = 0, mz = 0, m2 = 0;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (!alive.test(s)) continue;
            const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
            const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[s]);
            const Real ax = vx[r], ay = vy[r], az = vz[r];
            const Real a2 = ax * ax + ay * ay + az * az;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int f = (ids >> (8 * t)) & 0xff;
                const int nx_ = (adj >> (8 * ((t + 2) % 3))) & 0xff;
                const Real bx = sm.vpos[nx_][0], by = sm.vpos[nx_][1], bz = sm.vpos[nx_][2];
                const Real fnx = sm.pnx[f], fny = sm.pny[f], fnz = sm.pnz[f], fb = sm.pb[f];
                const Real nn = fnx * fnx + fny * fny + fnz * fnz;
                const Real sc = fb / nn;
                const Real qx = fnx * sc, qy = fny * sc, qz = fnz * sc;
                // det[q a b]
                const Real cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
                const Real det = qx * cx + qy * cy + qz * cz;
                const Real dv = det * (Real)(1.0 / 6.0);
                const Real sx = qx + ax + bx, sy = qy + ay + by, sz = qz + az + bz;
                vol += dv;
                mx += dv * sx;
                my += dv * sy;
                mz += dv * sz;
                m2 += dv * (qx * qx + qy * qy + qz * qz + a2 + bx * bx + by * by + bz * bz + sx * sx + sy * sy + sz * sz);
                // face area: 0.5 * (a - q) x (b - q) . n / |n|
                const Real ux = ax - qx, uy = ay - qy, uz = az - qz, wx = bx - qx, wy = by - qy, wz = bz - qz;
                const Real ar = (Real)0.5 * ((uy * wz - uz * wy) * fnx + (uz * wx - ux * wz) * fny + (ux * wy - uy * wx) * fnz) /
                                sqrt(nn);
                atomicAdd(&sm.u.tail.area[f], ar);
                sm.u.tail.first[f] = (int16_t)s;
            }
        }
        const double V = G.sum((double)vol);
        const double MX = G.sum((double)mx) * 0.25, MY = G.sum((double)my) * 0.25, MZ = G.sum((double)mz) * 0.25;
        const double M2 = G.sum((double)m2) * 0.05;
        G.sync();
        // neighbour keys: planes with a face of area above the threshold
        const double tau = Tol<Real>::area_rel * cbrt(V * V);
        for (int f = G.gl; f < np; f += T) {
            const int src = sm.psrc[f];
            const bool has = sm.u.tail.first[f] >= 0;
            int key = INT_MAX;
            if (src >= 0 && has && (double)sm.u.tail.area[f] > tau)
                key = A.index_space == VT_INDEX_ORIGINAL ? __float_as_int(sorted[src].w) : src;
            sm.u.tail.key[f] = key;
        }
        G.sync();
        if (G.gl == 0) {
            if (A.vol) A.vol[out_idx] = V;
            if (A.cen) {
                A.cen[3 * out_idx] = (double)pi.x + MX / V;
                A.cen[3 * out_idx + 1] = (double)pi.y + MY / V;
                A.cen[3 * out_idx + 2] = (double)pi.z + MZ / V;
            }
            if (A.m2) A.m2[out_idx] = M2;
        }
        if (!A.rec) return;
        uint8_t* rec = A.rec + (size_t)out_idx * A.rec_stride;
        int32_t* rnbr = reinterpret_cast<int32_t*>(rec + REC_NBR_OFF);
        int nn_total = 0;
        for (int f = G.gl; f < np; f += T) {
            const int key = sm.u.tail.key[f];
            if (key == INT_MAX) continue;
            int rank = 0;
            for (int g2 = 0; g2 < np; ++g2) rank += sm.u.tail.key[g2] < key ? 1 : 0;
            if (rank < REC_FACES) rnbr[rank] = key;
        }
        {
            int c = 0;
            for (int f = G.gl; f < np; f += T) c += sm.u.tail.key[f] != INT_MAX ? 1 : 0;
            nn_total = G.sum(c);
        }
        int nface = 0, nvtx = 0, nfv = 0;
        if (A.emit & VT_EMIT_GEOM) {
            nvtx = alive.count();
            // degrees by walking each face
            for (int f = G.gl; f < np; f += T) {
                int deg = 0;
                const int s0 = sm.u.tail.first[f];
                if (s0 >= 0) {
                    int cur = s0;
                    do {
                        const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[cur]);
                        const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[cur]);
                        int t = ((ids & 0xff) == (uint32_t)f) ? 0 : ((((ids >> 8) & 0xff) == (uint32_t)f) ? 1 : 2);
                        cur = (adj >> (8 * ((t + 2) % 3))) & 0xff;
                        ++deg;
                    } while (cur != s0 && deg <= VCAP);
                }
                sm.u.tail.deg[f] = (uint8_t)(deg > 255 ? 255 : deg);
            }
            G.sync();
            int32_t* rfn = reinterpret_cast<int32_t*>(rec + REC_FNBR_OFF);
            uint8_t* rdeg = rec + REC_FDEG_OFF;
            uint8_t* rfv = rec + REC_FVTX_OFF;
            double* rv = reinterpret_cast<double*>(rec + REC_VTX_OFF);
            for (int f = G.gl; f < np; f += T) {
                const int deg = sm.u.tail.deg[f];
                if (deg == 0) continue;
                int fi = 0, pos = 0;
                for (int g2 = 0; g2 < f; ++g2) {
                    const int dg = sm.u.tail.deg[g2];
                    fi += dg ? 1 : 0;
                    pos += dg;
                }
                if (fi >= REC_FACES || pos + deg > 3 * REC_VERTS) continue;
                const int src = sm.psrc[f];
                rfn[fi] = src < 0 ? src : (A.index_space == VT_INDEX_ORIGINAL ? __float_as_int(sorted[src].w) : src);
                rdeg[fi] = (uint8_t)deg;
                int cur = sm.u.tail.first[f];
                for (int t2 = 0; t2 < deg; ++t2) {
                    rfv[pos + t2] = (uint8_t)alive.rank(cur);
                    const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[cur]);
                    const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[cur]);
                    int t = ((ids & 0xff) == (uint32_t)f) ? 0 : ((((ids >> 8) & 0xff) == (uint32_t)f) ? 1 : 2);
                    cur = (adj >> (8 * ((t + 2) % 3))) & 0xff;
                }
            }
#pragma unroll
            for (int r = 0; r < VPL; ++r) {
                const int s = r * T + G.gl;
                if (alive.test(s)) {
                    const int li = alive.rank(s);
                    if (li < REC_VERTS) {
                        rv[3 * li] = (double)pi.x + (double)vx[r];
                        rv[3 * li + 1] = (double)pi.y + (double)vy[r];
                        rv[3 * li + 2] = (double)pi.z + (double)vz[r];
                    }
                }
            }
            int fc = 0, fvc = 0;
            for (int f = G.gl; f < np; f += T) {
                fc += sm.u.tail.deg[f] ? 1 : 0;
                fvc += sm.u.tail.deg[f];
            }
            nface = G.sum(fc);
            nfv = G.sum(fvc);
        }
        if (G.gl == 0) {
            bool over = nn_total > REC_FACES || nface > REC_FACES || nvtx > REC_VERTS || nfv > 3 * REC_VERTS;
            if (over) atomicAdd((int*)&st->record_overflow, 1);
            RecHeader* hd = reinterpret_cast<RecHeader*>(rec);
            hd->nnbr = over ? 0 : nn_total;
            hd->nface = over ? 0 : nface;
            hd->nvtx = over ? 0 : nvtx;
            hd->nfv = over ? 0 : nfv;
        }
        G.sync();
    }
};

// ---------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------
constexpr int CLIP_BLOCK = 128;

template <typename Real, int T, int VPL, int PCAP, bool ROBUST>
__global__ void __launch_bounds__(CLIP_BLOCK) k_clip(ClipArgs A)
{
    using C = Cell<Real, T, VPL, PCAP>;
    using S = typename C::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Group<T> G;
    S& sm = reinterpret_cast<S*>(smem_raw)[threadIdx.x / T];
    const int64_t gid = ((int64_t)blockIdx.x * CLIP_BLOCK + threadIdx.x) / T;
    const int64_t ngroups = ((int64_t)gridDim.x * CLIP_BLOCK) / T;
    const int k = A.k;
    const int Gr = A.g.G;

    uint32_t stamp = 0;
    for (int64_t c = gid; c < A.nq; c += ngroups) {
        const int q = A.queries ? A.queries[c] : (int)c;
        C cell(G, sm, A.sorted, A.g, A.st);
        cell.stamp = stamp;
        cell.pi = A.sorted[q];
        const int orig = __float_as_int(cell.pi.w);
        const int64_t out_idx = A.index_space == VT_INDEX_ORIGINAL ? (int64_t)orig : (int64_t)q;
        cell.init_box();
        int end = END_NEED_K;
        if (k > 0) {
            // neighbour list, nearest first
            const int32_t* nb = A.nbr + c * (int64_t)k;
            const Real* dd = reinterpret_cast<const Real*>(A.d2) + c * (int64_t)k;
            int m = 0;
            for (; m < k; ++m) {
                const int j = nb[m];
                if (j < 0) break;  // the list holds every other generator
                const Real dj = dd[m];
                if (cell.radius_ok(dj, j)) { end = END_VALID; break; }
                const int r = cell.clip_point(A.sorted[j], j);
                if (r == CLIP_OVERFLOW) { end = END_OVERFLOW; break; }
                if (r == CLIP_INCONSISTENT) { end = END_INCONSISTENT; break; }
            }
            if (m < k && end == END_NEED_K && nb[m] < 0) end = END_VALID;
            if (m == k && end == END_NEED_K && cell.radius_ok(dd[k - 1], nb[k - 1])) end = END_VALID;
        } else {
            // exhaustive: every generator closer than 2R, by a shell walk
            const float4 pq = cell.pi;
            const int ix = cell_coord(pq.x, A.g.lo[0], A.g.scale[0], Gr);
            const int iy = cell_coord(pq.y, A.g.lo[1], A.g.scale[1], Gr);
            const int iz = cell_coord(pq.z, A.g.lo[2], A.g.scale[2], Gr);
            int status = 0;
            auto scan_range = [&](int a, int b) {
                for (int base = a; base < b && status == 0; base += T) {
                    const int jj = base + G.gl;
                    float4 pc = make_float4(0, 0, 0, 0);
                    bool need = false;
                    if (jj < b && jj != q) {
                        pc = A.sorted[jj];
                        const double dx = (double)pc.x - (double)pq.x, dy = (double)pc.y - (double)pq.y,
                                     dz = (double)pc.z - (double)pq.z;
                        const double d2 = (dx * dx + dy * dy) + dz * dz;
                        need = 4.0 * (double)cell.R2 * (1.0 + 1e-5) > d2;
                    }
                    unsigned m = G.ballot(need);
                    while (m && status == 0) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const int j = G.bcast(jj, src);
                        const int r = cell.clip_point(A.sorted[j], j);
                        if (r == CLIP_OVERFLOW) status = END_OVERFLOW;
                        if (r == CLIP_INCONSISTENT) status = END_INCONSISTENT;
                    }
                }
            };
            for (int s = 0; status == 0; ++s) {
                for (int dx = -s; dx <= s && status == 0; ++dx) {
                    const int x = ix + dx;
                    if (x < 0 || x >= Gr) continue;
                    for (int dy = -s; dy <= s && status == 0; ++dy) {
                        const int y = iy + dy;
                        if (y < 0 || y >= Gr) continue;
                        const bool full = dx == -s || dx == s || dy == -s || dy == s;
                        if (full) {
                            const int z0 = max(iz - s, 0), z1 = min(iz + s, Gr - 1);
                            scan_range(A.cell_off[cell_id(x, y, z0, Gr)], A.cell_off[cell_id(x, y, z1, Gr) + 1]);
                        } else {
                            if (iz - s >= 0) {
                                const int cc = cell_id(x, y, iz - s, Gr);
                                scan_range(A.cell_off[cc], A.cell_off[cc + 1]);
                            }
                            if (iz + s < Gr) {
                                const int cc = cell_id(x, y, iz + s, Gr);
                                scan_range(A.cell_off[cc], A.cell_off[cc + 1]);
                            }
                        }
                    }
                }
                if (status) break;
                const bool covers = ix - s <= 0 && iy - s <= 0 && iz - s <= 0 && ix + s >= Gr - 1 &&
                                    iy + s >= Gr - 1 && iz + s >= Gr - 1;
                if (covers) { status = -1; break; }
                const double qc[3] = {(double)pq.x, (double)pq.y, (double)pq.z};
                const int ic[3] = {ix, iy, iz};
                double gap = 1e300;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (ic[a] - s > 0) gap = fmin(gap, qc[a] - ((double)A.g.lo[a] + (ic[a] - s) * A.g.cw[a]) - A.g.margin);
                    if (ic[a] + s + 1 < Gr)
                        gap = fmin(gap, ((double)A.g.lo[a] + (ic[a] + s + 1) * A.g.cw[a]) - qc[a] - A.g.margin);
                }
                if (gap > 0 && 4.0 * (double)cell.R2 * (1.0 + 1e-5) <= gap * gap) { status = -1; break; }
            }
            end = status == -1 ? END_VALID : status;
        }

        stamp = cell.stamp + 1;
        if (end == END_VALID) {
            cell.finish(out_idx, A, q);
        } else {
            if (G.gl == 0) {
                if (A.rec) {
                    RecHeader* hd = reinterpret_cast<RecHeader*>(A.rec + (size_t)out_idx * A.rec_stride);
                    hd->nnbr = hd->nface = hd->nvtx = hd->nfv = 0;
                }
                if (end == END_NEED_K && k > 0) {
                    const int slot = atomicAdd(A.ctr_next, 1);
                    A.fail_next[slot] = q;
                } else {
                    if (!ROBUST) {
                        if (end == END_OVERFLOW) atomicAdd(&A.st->capacity_events, 1ull);
                        else atomicAdd(&A.st->precision_events, 1ull);
                    }
                    const int slot = atomicAdd(A.ctr_robust, 1);
                    A.fail_robust[slot] = q;
                }
            }
            G.sync();
        }
    }
}

template <typename Real, int T, int VPL, int PCAP, bool ROBUST>
cudaError_t launch_variant(const ClipArgs& a, cudaStream_t s)
{
    using S = GroupSmem<Real, T * VPL, PCAP>;
    const size_t smem = sizeof(S) * (CLIP_BLOCK / T);
    auto kern = k_clip<Real, T, VPL, PCAP, ROBUST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int gpb = CLIP_BLOCK / T;
    int64_t blocks = (a.nq + gpb - 1) / gpb;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, CLIP_BLOCK, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

}  // namespace vt
