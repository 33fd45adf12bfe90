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
//  * planes n.x <= b in shared memory (SoA), with the source of each plane
//    (sorted index of the neighbour, or -1..-6 for the walls x-,x+,y-,y+,z-,z+);
//  * vertices in VCAP slots, all in shared memory. Lane s % T owns slot s
//    (row s / T) for the per-vertex steps (the sign pass of a cut reads its
//    rows' positions; keeping them in registers instead cost more spills
//    than the loads). Each slot holds its position, the three planes meeting
//    at the vertex,
//    (a, b, c), counter-clockwise seen from outside, and three adjacency
//    links: the vertex across the polyhedron edge between faces a&b, b&c and
//    c&a. A 128-bit mask marks the live slots (group-uniform).
//
// Clipping by a plane h: every lane tests its live vertices; removed vertices
// form a connected patch. Each edge (x -> y) of a removed vertex whose
// neighbour w across it survives is a boundary edge and yields one new vertex
// with planes (x, y, h) on the cut edge; its link across x&y is w, and the new
// vertices chain around h through start_of[x] / end_of[y] tables (each face
// x is cut at most once, so x starts exactly one boundary edge). New vertices
// take the lowest slots free before the clip (removed slots are freed after
// it), and their positions are solved from the three planes by the owners.
//
// Passes: a cell that needs a longer neighbour list saves its polyhedron
// (state) and the next pass resumes at the first unprocessed neighbour, so
// the k-doubling re-queue never repeats a clip; the exhaustive pass resumes
// from the k_max state and skips generators already in the list.
//
// FP32 form: planes, vertices and sign tests in float32. A sign test with
// |s| < 1e-6 |n| R is re-decided in FP64 from the vertex's three planes
// rebuilt in FP64 from the input points; the security-radius test is
// re-decided in FP64 (vertices re-solved in FP64) when it is within 1e-5
// relative of equality; volumes and moments accumulate per lane in float32 and
// across lanes in FP64. A topology inconsistency (a face cut twice) sends the
// cell to the robust FP64 variant.
#pragma once
#include <float.h>
#include <limits.h>

#include "vt_internal.cuh"

// rarely taken paths are out of line by default (smaller hot loop); building
// with -DVT_INLINE_RARE inlines them (no call-site register spills)
#ifdef VT_INLINE_RARE
#define VT_RARE __forceinline__
#else
#define VT_RARE __noinline__
#endif

namespace vt {

#ifdef VT_PROFILE
// section clocks and event counts of the clip kernels (diagnostic builds only):
// [8 * EXH + i], i = 0 cells, 1 setup cycles, 2 list/walk cycles, 3 clip
// cycles, 4 clip calls, 5 cuts, 6 finish cycles, 7 walk candidates; walk:
// 16 shells, 17 segment groups, 18 candidate batches, 19 raw candidates,
// 20 segment cycles, 21 candidate-test cycles, 22 survivor cycles (clips
// included), 23 batches without a survivor
static __device__ unsigned long long g_vt_prof[32];  // one copy per translation unit
#define VT_PROF_ADD(i, v) atomicAdd(&g_vt_prof[(i)], (unsigned long long)(v))
#else
#define VT_PROF_ADD(i, v) ((void)0)
#endif

namespace {

// ---------------------------------------------------------------------------
// slot masks of W 64-bit words (W = 1 for 64 slots, 2 for 128)
// ---------------------------------------------------------------------------
template <int W>
struct MaskW {
    static constexpr int W_ = W;
    uint64_t w[W];
    __device__ __forceinline__ bool test(int s) const
    {
        if (W == 1) return (w[0] >> s) & 1ull;
        return (w[s >> 6] >> (s & 63)) & 1ull;
    }
    __device__ __forceinline__ bool none() const
    {
        uint64_t o = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) o |= w[i];
        return o == 0;
    }
    __device__ __forceinline__ int count() const
    {
        int c = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) c += __popcll(w[i]);
        return c;
    }
    // number of set bits strictly below s
    __device__ __forceinline__ int rank(int s) const
    {
        if (W == 1) return __popcll(w[0] & ((1ull << s) - 1ull));
        if (s < 64) return __popcll(w[0] & ((1ull << s) - 1ull));
        return __popcll(w[0]) + __popcll(w[W - 1] & ((1ull << (s - 64)) - 1ull));
    }
    // 1 + highest set bit (0 if empty)
    __device__ __forceinline__ int top() const
    {
        if (W == 1) return w[0] ? 64 - __clzll(w[0]) : 0;
        return w[W - 1] ? 128 - __clzll(w[W - 1]) : (w[0] ? 64 - __clzll(w[0]) : 0);
    }
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int i = 0; i < W; ++i) w[i] = 0;
    }
    __device__ __forceinline__ void or_bits(uint64_t bits, int sh)
    {
        if (W == 1) w[0] |= bits << sh;
        else w[sh >> 6] |= bits << (sh & 63);
    }
};

template <int W>
__device__ __forceinline__ MaskW<W> mask_and(MaskW<W> a, MaskW<W> b)
{
#pragma unroll
    for (int i = 0; i < W; ++i) a.w[i] &= b.w[i];
    return a;
}
template <int W>
__device__ __forceinline__ MaskW<W> mask_or(MaskW<W> a, MaskW<W> b)
{
#pragma unroll
    for (int i = 0; i < W; ++i) a.w[i] |= b.w[i];
    return a;
}
template <int W>
__device__ __forceinline__ MaskW<W> mask_not(MaskW<W> a, int cap)
{
#pragma unroll
    for (int i = 0; i < W; ++i) {
        a.w[i] = ~a.w[i];
        const int lim = cap - 64 * i;
        if (lim <= 0) a.w[i] = 0;
        else if (lim < 64) a.w[i] &= (1ull << lim) - 1ull;
    }
    return a;
}
// position of the n-th (0-based) set bit of x, given popc(x) > n: a binary
// search on population counts
__device__ __forceinline__ int nth_bit32(uint32_t x, int n)
{
    int pos = 0, c = __popc(x & 0xffffu);
    if (n >= c) { n -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xffu);
    if (n >= c) { n -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xfu);
    if (n >= c) { n -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (n >= c) { n -= c; x >>= 2; pos += 2; }
    if (n >= (int)(x & 1u)) pos += 1;
    return pos;
}
// position of the i-th (0-based) set bit, or -1
template <int W>
__device__ __forceinline__ int nth_set(MaskW<W> m, int i)
{
#pragma unroll
    for (int h = 0; h < W; ++h) {
        const uint32_t lo = (uint32_t)m.w[h], hi = (uint32_t)(m.w[h] >> 32);
        const int cl = __popc(lo);
        if (i < cl) return h * 64 + nth_bit32(lo, i);
        i -= cl;
        const int ch = __popc(hi);
        if (i < ch) return h * 64 + 32 + nth_bit32(hi, i);
        i -= ch;
    }
    return -1;
}
// the bits of m at positions <= last
template <int W>
__device__ __forceinline__ MaskW<W> upto(MaskW<W> m, int last)
{
    MaskW<W> r = m;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const int lim = last - 64 * i;  // keep bits <= lim in word i
        if (lim < 0) r.w[i] = 0;
        else if (lim < 63) r.w[i] &= (1ull << (lim + 1)) - 1ull;
    }
    return r;
}
// rows of lane gl whose slot (r*T + gl) is set in m
template <int T, int VPL, int W>
__device__ __forceinline__ uint32_t lane_rows(MaskW<W> m, int gl)
{
    uint32_t b = 0;
#pragma unroll
    for (int r = 0; r < VPL; ++r) b |= (uint32_t)m.test(r * T + gl) << r;
    return b;
}
using Mask = MaskW<2>;

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

template <bool PER>
__device__ __forceinline__ P64 plane64(int src, const float4* __restrict__ sorted, float4 pi, const GridDesc& g)
{
    P64 p;
    if (src >= 0) {
        if (PER) {  // the image named by the entry's code
            const float4 pj = sorted[src & IMG_INDEX_MASK];
            int tx, ty, tz;
            img_t((int)((unsigned)src >> 24), tx, ty, tz);
            p.x = img_d64(pj.x, pi.x, tx, g.lo[0], g.hi[0]);
            p.y = img_d64(pj.y, pi.y, ty, g.lo[1], g.hi[1]);
            p.z = img_d64(pj.z, pi.z, tz, g.lo[2], g.hi[2]);
        } else {
            float4 pj = sorted[src];
            p.x = (double)pj.x - (double)pi.x;
            p.y = (double)pj.y - (double)pi.y;
            p.z = (double)pj.z - (double)pi.z;
        }
        p.b = 0.5 * ((p.x * p.x + p.y * p.y) + p.z * p.z);
    } else {
        const int w = -src - 1, axis = w >> 1, upper = w & 1;
        p.x = p.y = p.z = 0.0;
        const double pc = axis == 0 ? (double)pi.x : (axis == 1 ? (double)pi.y : (double)pi.z);
        const double v = upper ? 1.0 : -1.0;
        if (axis == 0) p.x = v; else if (axis == 1) p.y = v; else p.z = v;
        if (PER)  // the bisector with the own image one period away
            p.b = 0.5 * ((double)g.hi[axis] - (double)g.lo[axis]);
        else
            p.b = upper ? (double)g.hi[axis] - pc : pc - (double)g.lo[axis];
    }
    return p;
}

// 1 / x correctly rounded (the value of the IEEE division, without its
// general-purpose slow path)
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

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
    const Real inv = rcp(det);
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
    static constexpr int VCAP_ = VCAP;
    // Planes n.x <= b. In float32 the offset b of a bisector is |n|^2 / 2,
    // formed from n where it is needed (the expression of clip_point), and
    // the walls' offsets are kept apart: the footprint of a group sets the
    // shared memory of a block, and with it the L1 left to the clipper's
    // spilled registers. FP64 offsets are stored (the FP64 pipe is scarce).
    static constexpr bool STORE_B = sizeof(Real) == 8;
    Real pnx[PCAP], pny[PCAP], pnz[PCAP];
    Real pbs[STORE_B ? PCAP : 1];
    Real wall_b[8];         // offsets of the six walls (cube faces in a periodic box)
    int32_t psrc[PCAP];
    uint8_t vid[VCAP][4];   // planes a, b, c (ccw from outside)
    uint8_t vadj[VCAP][4];  // neighbour across a&b, b&c, c&a
    union {
        struct {  // one clip
            uint32_t start_of[PCAP];  // (stamp << 8) | slot
            uint32_t end_of[PCAP];
            uint16_t elist[VCAP];     // boundary edges of the current clip: slot | (edge << 8)
            uint8_t dlist[VCAP];      // slot of the new vertex of each boundary edge
            uint8_t vsrc[VCAP];       // removed vertex whose cut edge created the slot
        } ring;
        struct {  // the finish of a validated cell
            Real sc[PCAP];        // b / |n|^2 (the foot of the generator's perpendicular is n * sc); then
                                  // the neighbour key of the face, written by the plane's own lane
            int32_t first[PCAP];  // lowest live slot on the face (a face's walk starts there)
            int32_t deg[PCAP];    // live vertices on the face
        } tail;
    } u;
    __device__ __forceinline__ Real pb(int f) const
    {
        if (STORE_B) return pbs[f];
        const int src = psrc[f];
        if (src < 0) return wall_b[-src - 1];
        return (Real)0.5 * (pnx[f] * pnx[f] + pny[f] * pny[f] + pnz[f] * pnz[f]);
    }
    // (x, y, z, |v|^2) of each slot; the slots of dead vertices hold zeros,
    // so a plane test over all slots of the live rows needs no mask
    alignas(16) Real vpos[VCAP][4];
};

// a face's neighbour key in the slot of its plane's scale (bit patterns)
__device__ __forceinline__ void put_key(float* a, int f, int key) { a[f] = __int_as_float(key); }
__device__ __forceinline__ void put_key(double* a, int f, int key) { a[f] = __longlong_as_double((long long)key); }
__device__ __forceinline__ int get_key(const float* a, int f) { return __float_as_int(a[f]); }
__device__ __forceinline__ int get_key(const double* a, int f) { return (int)__double_as_longlong(a[f]); }

// vertex slot access: one 16-byte shared-memory access per float vertex
template <typename Real>
struct V4 { Real x, y, z, w; };
__device__ __forceinline__ V4<float> ldv(const float (*vp)[4], int s)
{
    const float4 t = *reinterpret_cast<const float4*>(vp[s]);
    return {t.x, t.y, t.z, t.w};
}
__device__ __forceinline__ V4<double> ldv(const double (*vp)[4], int s)
{
    const double2 a = *reinterpret_cast<const double2*>(vp[s]);
    const double2 b = *reinterpret_cast<const double2*>(vp[s] + 2);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void stv(float (*vp)[4], int s, float x, float y, float z)
{
    *reinterpret_cast<float4*>(vp[s]) = make_float4(x, y, z, x * x + y * y + z * z);
}
__device__ __forceinline__ void stv(double (*vp)[4], int s, double x, double y, double z)
{
    *reinterpret_cast<double2*>(vp[s]) = make_double2(x, y);
    *reinterpret_cast<double2*>(vp[s] + 2) = make_double2(z, x * x + y * y + z * z);
}


enum ClipResult { CLIP_NONE = 0, CLIP_CUT = 1, CLIP_OVERFLOW = 2, CLIP_INCONSISTENT = 3 };
enum CellEnd { END_VALID = 0, END_NEED_K = 1, END_OVERFLOW = 2, END_INCONSISTENT = 3 };

// A plane n.x <= b whose outside vertices (s = n.v - b > 0) all have s below
// on_plane_rel * |n| * R (R = cell radius) only touches the cell and is
// skipped: round-off of FP64 vertex positions at exactly degenerate inputs
// (lattices) must not cut slivers. Any other plane removes every vertex with
// s > 0. A 3x3 solve whose determinant is below cond_rel * |A||B||C| is replaced by
// interpolation along the cut edge.
template <typename Real>
struct Tol;
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

// ---------------------------------------------------------------------------
// saved polyhedron of a cell between passes (fixed stride per cell): the
// StateHdr, each plane's source, the topology and the vertex positions; the
// FP64 form also keeps its planes (forming them again on restore costs FP64
// operations), the FP32 form forms them again from the generators, exactly as
// clip_point formed them
// ---------------------------------------------------------------------------
template <typename Real, int VCAP, int PCAP>
struct StateLayout {
    static constexpr bool PLANES_KEPT = sizeof(Real) == 8;
    static constexpr size_t PLANES = (sizeof(StateHdr) + 31) / 32 * 32;                // Real[4][PCAP]
    static constexpr size_t PSRC = PLANES + (PLANES_KEPT ? 4 * sizeof(Real) * PCAP : 0);  // int32[PCAP]
    static constexpr size_t VID = PSRC + 4 * PCAP;                      // uint32[VCAP]
    static constexpr size_t VADJ = VID + 4 * VCAP;                      // uint32[VCAP]
    static constexpr size_t POS = (VADJ + 4 * VCAP + 15) / 16 * 16;     // Real[3][VCAP]
    static constexpr size_t BYTES = (POS + 3 * sizeof(Real) * VCAP + 255) / 256 * 256;
};

// ---------------------------------------------------------------------------
// rarely taken paths, kept out of line so the hot loop stays small
// ---------------------------------------------------------------------------

// FP64 re-decision of a sign test, the vertex re-solved from its planes:
// 0 inside or on the plane (s <= 0), 1 outside within the on-plane band
// (s^2 <= 1e-28 |n|^2 R^2), 2 outside beyond it
template <typename S>
__device__ VT_RARE int outside64(const S& sm, int s, P64 h, const float4* __restrict__ sorted, float4 pi,
                                      GridDesc g, double fx, double fy, double fz, double R2)
{
    const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
    const bool per = g.periodic != 0;  // out of line: the box kind is read here
    P64 A = per ? plane64<true>(sm.psrc[ids & 0xff], sorted, pi, g) : plane64<false>(sm.psrc[ids & 0xff], sorted, pi, g);
    P64 B = per ? plane64<true>(sm.psrc[(ids >> 8) & 0xff], sorted, pi, g)
                : plane64<false>(sm.psrc[(ids >> 8) & 0xff], sorted, pi, g);
    P64 C = per ? plane64<true>(sm.psrc[(ids >> 16) & 0xff], sorted, pi, g)
                : plane64<false>(sm.psrc[(ids >> 16) & 0xff], sorted, pi, g);
    double x, y, z;
    if (!vertex64(A, B, C, x, y, z)) { x = fx; y = fy; z = fz; }
    const double sv = (h.x * x + h.y * y) + h.z * z - h.b;
    if (!(sv > 0.0)) return 0;
    return sv * sv > ON_PLANE_REL2 * 2.0 * h.b * R2 ? 2 : 1;
}

// FP64 squared distance of slot s's vertex, re-solved from its planes
template <typename S>
__device__ VT_RARE double vertex_r2_64(const S& sm, int s, const float4* __restrict__ sorted, float4 pi,
                                            GridDesc g, double fx, double fy, double fz)
{
    const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
    const bool per = g.periodic != 0;
    P64 A = per ? plane64<true>(sm.psrc[ids & 0xff], sorted, pi, g) : plane64<false>(sm.psrc[ids & 0xff], sorted, pi, g);
    P64 B = per ? plane64<true>(sm.psrc[(ids >> 8) & 0xff], sorted, pi, g)
                : plane64<false>(sm.psrc[(ids >> 8) & 0xff], sorted, pi, g);
    P64 C = per ? plane64<true>(sm.psrc[(ids >> 16) & 0xff], sorted, pi, g)
                : plane64<false>(sm.psrc[(ids >> 16) & 0xff], sorted, pi, g);
    double x, y, z;
    if (!vertex64(A, B, C, x, y, z)) { x = fx; y = fy; z = fz; }
    return (x * x + y * y) + z * z;
}

// lowest plane id that no live vertex references (or -1)
template <int T, typename S, typename M>
__device__ VT_RARE int free_plane(const S& sm, M keep, int gl, unsigned gmask, int pcap, int vcap)
{
    uint64_t ref0 = 0, ref1 = 0;
    for (int s = gl; s < vcap; s += T) {
        if (!keep.test(s)) continue;
        const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int pid = (ids >> (8 * e)) & 0xff;
            if (pid < 64) ref0 |= 1ull << pid; else ref1 |= 1ull << (pid - 64);
        }
    }
#pragma unroll
    for (int o = T / 2; o >= 1; o >>= 1) {
        ref0 |= __shfl_xor_sync(gmask, ref0, o, T);
        ref1 |= __shfl_xor_sync(gmask, ref1, o, T);
    }
    return nth_set(mask_not(Mask{{ref0, ref1}}, pcap), 0);
}

// position of a new vertex by interpolation along its cut edge (the
// pre-clip vertex positions are in sm.vpos)
template <typename Real, typename S>
__device__ VT_RARE void interp_vertex(const S& sm, int s, Real nx, Real ny, Real nz, Real b, Real* xyz, DevStatus* st)
{
    const int v = vt_ck(sm.u.ring.vsrc[s], S::VCAP_, CK_SLOT, st), w = vt_ck(sm.vadj[s][0], S::VCAP_, CK_SLOT, st);
    const V4<Real> pv = ldv(sm.vpos, v), qv = ldv(sm.vpos, w);
    const Real px = pv.x, py = pv.y, pz = pv.z;
    const Real qx = qv.x, qy = qv.y, qz = qv.z;
    const Real sv = nx * px + ny * py + nz * pz - b, sw = nx * qx + ny * qy + nz * qz - b;
    Real t = sv - sw > (Real)0 ? sv / (sv - sw) : (Real)0.5;
    t = t < (Real)0 ? (Real)0 : (t > (Real)1 ? (Real)1 : t);
    xyz[0] = px + t * (qx - px);
    xyz[1] = py + t * (qy - py);
    xyz[2] = pz + t * (qz - pz);
}

// ---------------------------------------------------------------------------
// one cell: registers (positions, masks) + the group's shared memory
// ---------------------------------------------------------------------------
// PER: periodic box (images, the cube of one period) -- its own instantiation
template <typename Real, int T, int VPL, int PCAP, bool PER>
struct Cell {
    static constexpr int VCAP = T * VPL;
    using S = GroupSmem<Real, VCAP, PCAP>;
    using SL = StateLayout<Real, VCAP, PCAP>;
    using M = MaskW<(VCAP + 63) / 64>;

    // vertex positions live in the group's shared memory (sm.vpos): the
    // registers go to the clip's temporaries instead
    M alive;          // group-uniform
    int np;           // planes in use (ids < np)
    int rows;         // rows (slot / T) holding live slots
    uint32_t stamp;   // clip counter for the ring tables (keeps counting across cells)
    Real R2;          // max |v|^2 over live vertices
    float4 pi;

    __device__ __forceinline__ void get_row(const S& sm, int gl, int r, Real& x, Real& y, Real& z) const
    {
        const V4<Real> v = ldv(sm.vpos, r * T + gl);
        x = v.x;
        y = v.y;
        z = v.z;
    }

    __device__ __forceinline__ void update_rows() { rows = (alive.top() + T - 1) / T; }

    __device__ __forceinline__ void update_r2(const Group<T>& G, const S& sm)
    {
        // (dead slots hold zeros: every slot of the live rows is read)
        Real m = 0;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            if (r < rows) {
                const Real d = sm.vpos[r * T + G.gl][3];
                m = d > m ? d : m;
            }
        }
        R2 = G.max(m);
    }

    // axis-aligned bounding box of the live vertices (local frame), for the
    // exhaustive walk's support test
    __device__ __forceinline__ void bbox(const Group<T>& G, const S& sm, float* lo3, float* hi3) const
    {
        // every slot of the live rows is read: dead slots hold the origin (the
        // generator), which the cell contains, so the box is the same
        float l0 = FLT_MAX, l1 = FLT_MAX, l2 = FLT_MAX, h0 = -FLT_MAX, h1 = -FLT_MAX, h2 = -FLT_MAX;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (r < rows) {
                const V4<Real> v = ldv(sm.vpos, s);
                const float x = (float)v.x, y = (float)v.y, z = (float)v.z;
                l0 = fminf(l0, x); h0 = fmaxf(h0, x);
                l1 = fminf(l1, y); h1 = fmaxf(h1, y);
                l2 = fminf(l2, z); h2 = fmaxf(h2, z);
            }
        }
#pragma unroll
        for (int o = T / 2; o >= 1; o >>= 1) {
            l0 = fminf(l0, __shfl_xor_sync(G.mask, l0, o, T)); h0 = fmaxf(h0, __shfl_xor_sync(G.mask, h0, o, T));
            l1 = fminf(l1, __shfl_xor_sync(G.mask, l1, o, T)); h1 = fmaxf(h1, __shfl_xor_sync(G.mask, h1, o, T));
            l2 = fminf(l2, __shfl_xor_sync(G.mask, l2, o, T)); h2 = fmaxf(h2, __shfl_xor_sync(G.mask, h2, o, T));
        }
        lo3[0] = l0; lo3[1] = l1; lo3[2] = l2;
        hi3[0] = h0; hi3[1] = h1; hi3[2] = h2;
    }

    // the box's corners lo, hi in the frame of pi
    __device__ __forceinline__ void box_of(const GridDesc& grid, Real& lx, Real& ly, Real& lz, Real& hx, Real& hy,
                                           Real& hz) const
    {
        if (PER) {
            hx = (Real)(0.5 * ((double)grid.hi[0] - (double)grid.lo[0]));
            hy = (Real)(0.5 * ((double)grid.hi[1] - (double)grid.lo[1]));
            hz = (Real)(0.5 * ((double)grid.hi[2] - (double)grid.lo[2]));
            lx = -hx;
            ly = -hy;
            lz = -hz;
        } else {
            const Real px = (Real)pi.x, py = (Real)pi.y, pz = (Real)pi.z;
            lx = (Real)grid.lo[0] - px;
            ly = (Real)grid.lo[1] - py;
            lz = (Real)grid.lo[2] - pz;
            hx = (Real)grid.hi[0] - px;
            hy = (Real)grid.hi[1] - py;
            hz = (Real)grid.hi[2] - pz;
        }
    }

    // wall w (x-, x+, y-, y+, z-, z+) as plane f of the group
    __device__ __forceinline__ void set_wall(S& sm, int f, int w, Real lx, Real ly, Real lz, Real hx, Real hy,
                                             Real hz) const
    {
        const int axis = w >> 1, upper = w & 1;
        const Real one = upper ? (Real)1 : (Real)-1;
        sm.pnx[f] = axis == 0 ? one : (Real)0;
        sm.pny[f] = axis == 1 ? one : (Real)0;
        sm.pnz[f] = axis == 2 ? one : (Real)0;
        const Real lo_a = axis == 0 ? lx : (axis == 1 ? ly : lz);
        const Real hi_a = axis == 0 ? hx : (axis == 1 ? hy : hz);
        sm.wall_b[w] = upper ? hi_a : -lo_a;
        if (S::STORE_B) sm.pbs[f] = upper ? hi_a : -lo_a;
        sm.psrc[f] = -(w + 1);
    }

    // the box [lo, hi) in the frame of pi: walls 0..5, corners in slots 0..7;
    // in a periodic box the cube [-L/2, L/2] (the bisectors of pi's own images)
    __device__ __forceinline__ void init_box(const Group<T>& G, S& sm, const GridDesc& grid)
    {
        Real lx, ly, lz, hx, hy, hz;
        box_of(grid, lx, ly, lz, hx, hy, hz);
        if (G.gl < 6) set_wall(sm, G.gl, G.gl, lx, ly, lz, hx, hy, hz);
        if (G.gl < 8) {
            // corner c = 4 sx + 2 sy + sz; planes (x, y, z) in ccw order, swapped
            // when an odd number of its walls are lower walls (mirror image)
            const int c = G.gl, sx = (c >> 2) & 1, sy = (c >> 1) & 1, sz = c & 1;
            int p0 = sx, p1 = 2 + sy, p2 = 4 + sz;
            if (((1 - sx) + (1 - sy) + (1 - sz)) & 1) { const int t = p1; p1 = p2; p2 = t; }
            *reinterpret_cast<uint32_t*>(sm.vid[c]) = (uint32_t)p0 | ((uint32_t)p1 << 8) | ((uint32_t)p2 << 16);
            // neighbour across (P[e], P[e+1]): flip the axis of the third plane
            const uint32_t a0 = c ^ (4 >> (p2 >> 1)), a1 = c ^ (4 >> (p0 >> 1)), a2 = c ^ (4 >> (p1 >> 1));
            *reinterpret_cast<uint32_t*>(sm.vadj[c]) = a0 | (a1 << 8) | (a2 << 16);
        }
        alive.clear();
        alive.w[0] = 0xffull;
        np = 6;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {  // the corners in slots 0..7, zeros elsewhere
            const int c = r * T + G.gl;
            if (c < 8)
                stv(sm.vpos, c, ((c >> 2) & 1) ? hx : lx, ((c >> 1) & 1) ? hy : ly, (c & 1) ? hz : lz);
            else
                stv(sm.vpos, c, (Real)0, (Real)0, (Real)0);
        }
        update_rows();
        G.sync();
        update_r2(G, sm);
    }

    // ---- save / restore between passes ------------------------------------
    __device__ __forceinline__ void save(const Group<T>& G, const S& sm, uint8_t* st, double last_d2,
                                         int last_orig) const
    {
        int32_t* ps = reinterpret_cast<int32_t*>(st + SL::PSRC);
        Real* pl = reinterpret_cast<Real*>(st + SL::PLANES);
        for (int f = G.gl; f < np; f += T) {
            ps[f] = sm.psrc[f];
            if (SL::PLANES_KEPT) {
                pl[f] = sm.pnx[f];
                pl[PCAP + f] = sm.pny[f];
                pl[2 * PCAP + f] = sm.pnz[f];
                pl[3 * PCAP + f] = sm.pb(f);
            }
        }
        uint32_t* vi = reinterpret_cast<uint32_t*>(st + SL::VID);
        uint32_t* va = reinterpret_cast<uint32_t*>(st + SL::VADJ);
        Real* pos = reinterpret_cast<Real*>(st + SL::POS);
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (r < rows && alive.test(s)) {
                vi[s] = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
                va[s] = *reinterpret_cast<const uint32_t*>(sm.vadj[s]);
                const V4<Real> v = ldv(sm.vpos, s);
                pos[s] = v.x;
                pos[VCAP + s] = v.y;
                pos[2 * VCAP + s] = v.z;
            }
        }
        float lo3[3], hi3[3];
        bbox(G, sm, lo3, hi3);
        if (G.gl == 0) {
            StateHdr* h = reinterpret_cast<StateHdr*>(st);
#pragma unroll
            for (int a = 0; a < 3; ++a) { h->bb_lo[a] = lo3[a]; h->bb_hi[a] = hi3[a]; }
            h->alive[0] = alive.w[0];
            h->alive[1] = M::W_ == 2 ? alive.w[M::W_ - 1] : 0ull;
            h->np = np;
            h->last_orig = last_orig;
            h->R2 = (double)R2;
            h->last_d2 = last_d2;
        }
    }

    __device__ __forceinline__ void restore(const Group<T>& G, S& sm, const uint8_t* st, double& last_d2,
                                            int& last_orig, const float4* __restrict__ sorted, const GridDesc& grid)
    {
        const StateHdr* h = reinterpret_cast<const StateHdr*>(st);
        alive.w[0] = h->alive[0];
        if (M::W_ == 2) alive.w[M::W_ - 1] = h->alive[1];
        np = h->np;
        R2 = (Real)h->R2;
        last_d2 = h->last_d2;
        last_orig = h->last_orig;
        const int32_t* ps = reinterpret_cast<const int32_t*>(st + SL::PSRC);
        Real lx, ly, lz, hx, hy, hz;
        box_of(grid, lx, ly, lz, hx, hy, hz);
        const Real* pl = reinterpret_cast<const Real*>(st + SL::PLANES);
        for (int f = G.gl; f < np; f += T) {
            const int src = ps[f];
            if (SL::PLANES_KEPT) {
                sm.pnx[f] = pl[f];
                sm.pny[f] = pl[PCAP + f];
                sm.pnz[f] = pl[2 * PCAP + f];
                if (S::STORE_B) sm.pbs[f] = pl[3 * PCAP + f];
                if (src < 0) sm.wall_b[-src - 1] = pl[3 * PCAP + f];
                sm.psrc[f] = src;
                continue;
            }
            // each plane formed again from its source, exactly as when it cut
            if (src < 0) {
                set_wall(sm, f, -src - 1, lx, ly, lz, hx, hy, hz);
            } else {
                Real nx, ny, nz;
                normal_of(sorted[img_index_t<PER>(src)], src, grid, nx, ny, nz);
                sm.pnx[f] = nx;
                sm.pny[f] = ny;
                sm.pnz[f] = nz;
                if (S::STORE_B) sm.pbs[f] = (Real)0.5 * (nx * nx + ny * ny + nz * nz);
                sm.psrc[f] = src;
            }
        }
        update_rows();
        const uint32_t* vi = reinterpret_cast<const uint32_t*>(st + SL::VID);
        const uint32_t* va = reinterpret_cast<const uint32_t*>(st + SL::VADJ);
        const Real* pos = reinterpret_cast<const Real*>(st + SL::POS);
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            if (r < rows && alive.test(s)) {
                *reinterpret_cast<uint32_t*>(sm.vid[s]) = vi[s];
                *reinterpret_cast<uint32_t*>(sm.vadj[s]) = va[s];
                stv(sm.vpos, s, pos[s], pos[VCAP + s], pos[2 * VCAP + s]);
            } else {
                stv(sm.vpos, s, (Real)0, (Real)0, (Real)0);
            }
        }
        G.sync();
    }

    // true when no generator at squared distance >= dj can cut the cell
    __device__ __forceinline__ bool radius_ok(const Group<T>& G, const S& sm, Real dj, int jsrc,
                                              const float4* __restrict__ sorted, const GridDesc& grid, DevStatus* st)
    {
        if (!Tol<Real>::fp32) return (Real)4 * R2 <= dj;
        const float lhs = 4.0f * (float)R2, rhs = (float)dj;
        if (lhs <= rhs * (1.0f - 1e-5f)) return true;
        if (lhs > rhs * (1.0f + 1e-5f)) return false;
        // within 1e-5 of equality: decide in FP64, every vertex re-solved in FP64
        if (G.gl == 0) atomicAdd(&st->fp64_rechecks, 1ull);
        const double d64 = jsrc >= 0 ? 2.0 * plane64<PER>(jsrc, sorted, pi, grid).b : (double)dj;
        double m = 0;
        for (uint32_t rm = lane_rows<T, VPL>(alive, G.gl); rm; rm &= rm - 1) {
            const int r = __ffs(rm) - 1;
            Real fx, fy, fz;
            get_row(sm, G.gl, r, fx, fy, fz);
            const double d = vertex_r2_64(sm, r * T + G.gl, sorted, pi, grid, (double)fx, (double)fy, (double)fz);
            m = d > m ? d : m;
        }
        return 4.0 * G.max(m) <= d64;
    }

    // clip by n.x <= b (plane source src)
    __device__ __forceinline__ int clip(const Group<T>& G, S& sm, Real nx, Real ny, Real nz, Real b, int src,
                                        const float4* __restrict__ sorted, const GridDesc& grid, DevStatus* st)
    {
        // The on-plane rule applies to the cut as a whole: a plane whose
        // outside vertices all lie within the on-plane band (|s| below
        // 1e-14 |n| R, FP64 round-off at exactly degenerate vertices) only
        // touches the cell and is skipped; any other plane cuts every vertex
        // strictly outside it (s > 0). Keeping a vertex inside the band while
        // cutting the ones beyond it would split the outside set and break
        // the ring of the new face.
        M out;
        out.clear();
        uint32_t myout = 0, mynear = 0, myfar = 0;
        const double tol2 = Tol<Real>::fp32 ? 0.0 : ON_PLANE_REL2 * 2.0 * (double)b * (double)R2;
        const float near2 = Tol<Real>::fp32 ? 2e-12f * (float)b * (float)R2 : 0.0f;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            if (r < rows) {
                const int s = r * T + G.gl;
                const V4<Real> v = ldv(sm.vpos, s);
                const Real sv = nx * v.x + ny * v.y + nz * v.z - b;
                const bool al = alive.test(s);
                const bool o = al && sv > (Real)0;
                if (Tol<Real>::fp32) {
                    // beyond the FP32 recheck band an outside vertex is far outside
                    if (al && (float)sv * (float)sv < near2) mynear |= 1u << r;
                    else myfar |= (uint32_t)o << r;
                } else {
                    myfar |= (uint32_t)(o && (double)sv * (double)sv > tol2) << r;
                }
                myout |= (uint32_t)o << r;
                out.or_bits((uint64_t)G.ballot(o), r * T);
            }
        }
        if (Tol<Real>::fp32 && G.any(mynear != 0)) {
            // re-decide the near-zero tests in FP64
            const P64 h = plane64<PER>(src, sorted, pi, grid);
            for (uint32_t m = mynear; m; m &= m - 1) {
                const int r = __ffs(m) - 1;
                Real fx, fy, fz;
                get_row(sm, G.gl, r, fx, fy, fz);
                const int o = outside64(sm, r * T + G.gl, h, sorted, pi, grid, (double)fx, (double)fy, (double)fz,
                                        (double)R2);
                myout = o ? (myout | (1u << r)) : (myout & ~(1u << r));
                if (o == 2) myfar |= 1u << r;
                atomicAdd(&st->fp64_rechecks, 1ull);
            }
            out.clear();
#pragma unroll
            for (int r = 0; r < VPL; ++r)
                if (r < rows) out.or_bits((uint64_t)G.ballot((myout >> r) & 1u), r * T);
        }
        if (out.none() || !G.any(myfar != 0)) return CLIP_NONE;
        const M keep = mask_and(alive, mask_not(out, VCAP));
        if (keep.none()) {  // the generator itself is always inside
            if (G.gl == 0) atomicAdd(&st->detail[0], 1u);
            return CLIP_INCONSISTENT;
        }
        // plane id for h
        int h = np;
        if (np >= PCAP) {
            h = free_plane<T>(sm, keep, G.gl, G.mask, PCAP, VCAP);
            if (h < 0) {
                if (G.gl == 0) atomicAdd(&st->detail[1], 1u);
                return CLIP_OVERFLOW;
            }
        }
        // boundary edges of the removed patch: edge e of a removed vertex whose
        // neighbour across it survives (bit 3r+e of myedge)
        // (predicated, no branch: every lane reads its rows' links, and the
        // bits of the rows it does not remove stay clear)
        uint32_t myedge = 0;
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            if (r < rows) {
                const bool o = (myout >> r) & 1u;
                const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[r * T + G.gl]);
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    const int w = o ? vt_ck((adj >> (8 * e)) & 0xff, VCAP, CK_SLOT, st) : 0;
                    myedge |= (uint32_t)(o && !out.test(w)) << (3 * r + e);
                }
            }
        }
        int total;
        int idx = G.scan(__popc(myedge), total);
        // new vertices go to slots that were free before this clip, so the
        // removed vertices' topology stays readable until the ring is closed;
        // dlist[i] = the i-th free slot (the slot of the i-th new vertex)
        const M freem = mask_not(alive, VCAP);
        if (total > freem.count()) {
            if (G.gl == 0) atomicAdd(&st->detail[2], 1u);
            return CLIP_OVERFLOW;
        }
#pragma unroll
        for (int r = 0; r < VPL; ++r) {
            const int s = r * T + G.gl;
            const int k = freem.rank(s);
            if (freem.test(s) && k < total) sm.u.ring.dlist[k] = (uint8_t)s;
        }
        // this lane's boundary edges in bit order (a fixed, unrolled loop of
        // predicated stores: no per-lane trip count)
#pragma unroll
        for (int bit = 0; bit < 3 * VPL; ++bit) {
            if ((myedge >> bit) & 1u) {
                sm.u.ring.elist[vt_ck(idx, VCAP, CK_EDGE, st)] = (uint16_t)(((bit / 3) * T + G.gl) | ((bit % 3) << 8));
                ++idx;
            }
        }
        // the plane h: every lane stores the same values (no lane-0 branch)
        sm.pnx[h] = nx;
        sm.pny[h] = ny;
        sm.pnz[h] = nz;
        sm.psrc[h] = src;
        if (S::STORE_B) sm.pbs[h] = b;
        ++stamp;
        const uint32_t tag = stamp << 8;
        G.sync();
        // one boundary edge per lane: the new vertex (x, y, h) on the cut edge
        for (int i = G.gl; i < total; i += T) {
            const uint32_t ev = sm.u.ring.elist[i];
            const int s = vt_ck(ev & 0xff, VCAP, CK_SLOT, st), e = vt_ck(ev >> 8, 3, CK_EDGE, st);
            const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
            const int w = vt_ck(sm.vadj[s][e], VCAP, CK_SLOT, st);
            const int x = vt_ck((ids >> (8 * e)) & 0xff, PCAP, CK_PLANE, st);
            const int y = vt_ck((ids >> (8 * (e == 2 ? 0 : e + 1))) & 0xff, PCAP, CK_PLANE, st);
            const int d = vt_ck(sm.u.ring.dlist[i], VCAP, CK_SLOT, st);
            *reinterpret_cast<uint32_t*>(sm.vid[d]) = (uint32_t)x | ((uint32_t)y << 8) | ((uint32_t)h << 16);
            sm.vadj[d][0] = (uint8_t)w;
            sm.u.ring.vsrc[d] = (uint8_t)s;
            sm.u.ring.start_of[x] = tag | (uint32_t)d;
            sm.u.ring.end_of[y] = tag | (uint32_t)d;
            // the survivor w: its link across y&x now points to d
            const uint32_t wid = *reinterpret_cast<const uint32_t*>(sm.vid[w]);
            const int w0 = wid & 0xff, w1 = (wid >> 8) & 0xff;
            const int e2 = (w0 == y && w1 == x) ? 0 : ((w1 == y) ? 1 : 2);
            sm.vadj[w][e2] = (uint8_t)d;
        }
        G.sync();
        // close the ring around h and solve the new positions
        bool bad = false, need = false;
        for (int i = G.gl; i < total; i += T) {
            const int d = vt_ck(sm.u.ring.dlist[i], VCAP, CK_SLOT, st);
            const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[d]);
            const int x = vt_ck(ids & 0xff, PCAP, CK_PLANE, st), y = vt_ck((ids >> 8) & 0xff, PCAP, CK_PLANE, st);
            const uint32_t so = sm.u.ring.start_of[y], eo = sm.u.ring.end_of[x];
            if (VT_CHECKED) {
                vt_ck(so & 0xff, VCAP, CK_SLOT, st);
                vt_ck(eo & 0xff, VCAP, CK_SLOT, st);
            }
            if ((so & ~0xffu) != tag || (eo & ~0xffu) != tag || sm.u.ring.start_of[x] != (tag | (uint32_t)d))
                bad = true;
            sm.vadj[d][1] = (uint8_t)(so & 0xff);
            sm.vadj[d][2] = (uint8_t)(eo & 0xff);
            Real px, py, pz;
            if (solve3<Real>(sm.pnx[x], sm.pny[x], sm.pnz[x], sm.pb(x), sm.pnx[y], sm.pny[y], sm.pnz[y], sm.pb(y), nx,
                             ny, nz, b, px, py, pz, (Real)Tol<Real>::cond_rel)) {
                stv(sm.vpos, d, px, py, pz);
            } else {
                sm.vpos[d][0] = (Real)NAN;  // marks an interpolated vertex
                need = true;
            }
        }
        if (G.any(bad)) {
            if (G.gl == 0) atomicAdd(&st->detail[3], 1u);
            return CLIP_INCONSISTENT;
        }
        if (G.any(need)) {
            // ill-conditioned solves: interpolate along the cut edge from the
            // pre-clip positions (the new slots were free, so no overlap)
            if (G.gl == 0) atomicAdd(&st->detail[4], 1u);
            G.sync();
            for (int i = G.gl; i < total; i += T) {
                const int d = vt_ck(sm.u.ring.dlist[i], VCAP, CK_SLOT, st);
                if (isnan(sm.vpos[d][0])) {
                    Real xyz[3];
                    interp_vertex<Real>(sm, d, nx, ny, nz, b, xyz, st);
                    stv(sm.vpos, d, xyz[0], xyz[1], xyz[2]);
                }
            }
        }
        // the removed vertices' slots become zeros (read by whole-row plane
        // tests); the interpolation above still needed their positions
#pragma unroll
        for (int r = 0; r < VPL; ++r)
            if ((myout >> r) & 1u) stv(sm.vpos, r * T + G.gl, (Real)0, (Real)0, (Real)0);
        if (h == np) ++np;
        M newm;
        newm.clear();
        if (total > 0) newm = upto(freem, sm.u.ring.dlist[total - 1]);
        alive = mask_or(keep, newm);
        update_rows();
        G.sync();
        update_r2(G, sm);
        return CLIP_CUT;
    }

    // the bisector normal n = p_j - p_i (the image named by j's code in a
    // periodic box), in the arithmetic of the form
    __device__ __forceinline__ void normal_of(float4 pj, int j, const GridDesc& grid, Real& nx, Real& ny,
                                              Real& nz) const
    {
        // j packs the image code; an unshifted image (almost every entry) takes
        // the walled arithmetic (j is uniform over the group: no divergence)
        const int code = PER ? (int)((unsigned)j >> 24) : IMG_NONE;
        if (PER && code != IMG_NONE) {
            if (Tol<Real>::fp32) {
                const float3 o = img_off(pi, pj, code, grid);
                nx = (Real)o.x;
                ny = (Real)o.y;
                nz = (Real)o.z;
            } else {
                int tx, ty, tz;
                img_t(code, tx, ty, tz);
                nx = (Real)img_d64(pj.x, pi.x, tx, grid.lo[0], grid.hi[0]);
                ny = (Real)img_d64(pj.y, pi.y, ty, grid.lo[1], grid.hi[1]);
                nz = (Real)img_d64(pj.z, pi.z, tz, grid.lo[2], grid.hi[2]);
            }
        } else if (Tol<Real>::fp32) {
            nx = (Real)(pj.x - pi.x);
            ny = (Real)(pj.y - pi.y);
            nz = (Real)(pj.z - pi.z);
        } else {
            nx = (Real)pj.x - (Real)pi.x;
            ny = (Real)pj.y - (Real)pi.y;
            nz = (Real)pj.z - (Real)pi.z;
        }
    }

    __device__ __forceinline__ int clip_point(const Group<T>& G, S& sm, float4 pj, int j,
                                              const float4* __restrict__ sorted, const GridDesc& grid, DevStatus* st)
    {
        Real nx, ny, nz;
        normal_of(pj, j, grid, nx, ny, nz);
        const Real b = (Real)0.5 * (nx * nx + ny * ny + nz * nz);
        return clip(G, sm, nx, ny, nz, b, j, sorted, grid, st);
    }

    // Per-lane test of one plane n.x <= |n|^2 / 2 (n = pj - pi) against every
    // live vertex, positions read from sm.vpos: false only when each vertex is
    // inside by more than 1e-5 |n| R, beyond the band the sign test re-decides
    // in FP64, so a plane that fails cannot cut and clip() would do nothing.
    // (Every slot of the live rows is read, four at a time: dead slots hold
    // zeros, which pass only when lim < 0, a harmless extra clip.)
    __device__ __forceinline__ bool reaches(const S& sm, float nx, float ny, float nz) const
    {
        const float nn = nx * nx + ny * ny + nz * nz;
        const float lim = 0.5f * nn - 1e-5f * sqrtf(nn * (float)R2) - 1e-30f;
        if (!Tol<Real>::fp32) {  // FP64 slots are twice as wide: only the live ones
#pragma unroll
            for (int w = 0; w < M::W_; ++w) {
                for (uint64_t m = alive.w[w]; m; m &= m - 1ull) {
                    const V4<Real> v = ldv(sm.vpos, w * 64 + __ffsll((long long)m) - 1);
                    if (nx * (float)v.x + ny * (float)v.y + nz * (float)v.z > lim) return true;
                }
            }
            return false;
        }
        const int ns = rows * T;
        for (int s = 0; s < ns; s += 4) {
            const V4<Real> a = ldv(sm.vpos, s), b = ldv(sm.vpos, s + 1), c = ldv(sm.vpos, s + 2),
                           d = ldv(sm.vpos, s + 3);
            const float da = nx * (float)a.x + ny * (float)a.y + nz * (float)a.z;
            const float db = nx * (float)b.x + ny * (float)b.y + nz * (float)b.z;
            const float dc = nx * (float)c.x + ny * (float)c.y + nz * (float)c.z;
            const float dd = nx * (float)d.x + ny * (float)d.y + nz * (float)d.z;
            if (fmaxf(fmaxf(da, db), fmaxf(dc, dd)) > lim) return true;
        }
        return false;
    }

};

// ---------------------------------------------------------------------------
// moments, neighbours and geometry of a validated cell (shared memory only)
// ---------------------------------------------------------------------------
template <typename Real, int T, int VCAP, int PCAP, typename M, bool PER>
__device__ VT_RARE void finish_cell(GroupSmem<Real, VCAP, PCAP>& sm, M alive, int np, float4 pi, int gl,
                                         unsigned gmask, int64_t out_idx, const ClipArgs& A)
{
    // per plane: q_f = n sc, the foot of the perpendicular from the
    // generator onto it (the apex of the face's fan); counters (the union's
    // other half is free: its size sets the shared memory per block, and with
    // it the L1 left to the clipper's spills)
    for (int f = gl; f < np; f += T) {
        const Real fnx = sm.pnx[f], fny = sm.pny[f], fnz = sm.pnz[f];
        sm.u.tail.sc[f] = sm.pb(f) / (fnx * fnx + fny * fny + fnz * fnz);
        sm.u.tail.first[f] = INT_MAX;
        sm.u.tail.deg[f] = 0;
    }
    __syncwarp(gmask);
    // per (vertex, face) terms: tetrahedron (0, q_f, v, next(v around f));
    // each face's degree and lowest live slot
    Real vol = 0, mx = 0, my = 0, mz = 0, m2 = 0;
    for (int s = gl; s < VCAP; s += T) {
        if (!alive.test(s)) continue;
        const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[s]);
        const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[s]);
        const V4<Real> va = ldv(sm.vpos, s);
        const Real ax = va.x, ay = va.y, az = va.z;
        const Real a2 = va.w;
        for (int t = 0; t < 3; ++t) {
            const int f = vt_ck((ids >> (8 * t)) & 0xff, PCAP, CK_PLANE, A.st);
            const int nv = vt_ck((adj >> (8 * (t == 0 ? 2 : t - 1))) & 0xff, VCAP, CK_SLOT, A.st);
            const V4<Real> vb = ldv(sm.vpos, nv);
            const Real bx = vb.x, by = vb.y, bz = vb.z;
            const Real sc = sm.u.tail.sc[f];
            const Real qx = sm.pnx[f] * sc, qy = sm.pny[f] * sc, qz = sm.pnz[f] * sc;
            const Real cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
            const Real dv = (qx * cx + qy * cy + qz * cz) * (Real)(1.0 / 6.0);
            const Real sx = qx + ax + bx, sy = qy + ay + by, sz = qz + az + bz;
            vol += dv;
            mx += dv * sx;
            my += dv * sy;
            mz += dv * sz;
            m2 += dv * (qx * qx + qy * qy + qz * qz + a2 + bx * bx + by * by + bz * bz + sx * sx + sy * sy + sz * sz);
            atomicMin(&sm.u.tail.first[f], s);
            atomicAdd(&sm.u.tail.deg[f], 1);
        }
    }
    // FP64 sums across the lanes by reduce-scatter: the five sums (padded to
    // eight slots) are halved between partners at the first three levels, so
    // a group of 32 lanes adds 9 times instead of 25 (the FP64 pipe is 1/64
    // of FP32); lane 4 b1 T/8 ... holds slot 4 b1 + 2 b2 + b3 at the end
    double w;
    {
        const double s0[8] = {(double)vol, (double)mx, (double)my, (double)mz, (double)m2, 0.0, 0.0, 0.0};
        double t4[4], t2[2];
        const bool hi1 = (gl & (T / 2)) != 0, hi2 = (gl & (T / 4)) != 0, hi3 = (gl & (T / 8)) != 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double send = hi1 ? s0[i] : s0[4 + i];
            t4[i] = (hi1 ? s0[4 + i] : s0[i]) + __shfl_xor_sync(gmask, send, T / 2, T);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double send = hi2 ? t4[i] : t4[2 + i];
            t2[i] = (hi2 ? t4[2 + i] : t4[i]) + __shfl_xor_sync(gmask, send, T / 4, T);
        }
        w = (hi3 ? t2[1] : t2[0]) + __shfl_xor_sync(gmask, hi3 ? t2[0] : t2[1], T / 8, T);
#pragma unroll
        for (int o = T / 16; o >= 1; o >>= 1) w += __shfl_xor_sync(gmask, w, o, T);
    }
    const double V = __shfl_sync(gmask, w, 0, T);
    const double MX = 0.25 * __shfl_sync(gmask, w, T / 8, T);
    const double MY = 0.25 * __shfl_sync(gmask, w, T / 4, T);
    const double MZ = 0.25 * __shfl_sync(gmask, w, T / 4 + T / 8, T);
    const double M2 = 0.05 * __shfl_sync(gmask, w, T / 2, T);
    __syncwarp(gmask);  // the degrees and lowest slots are complete
    if (gl == 0) {
        if (A.vol) A.vol[out_idx] = V;
        if (A.cen) {
            const double iv = 1.0 / V;
            A.cen[3 * out_idx] = (double)pi.x + MX * iv;
            A.cen[3 * out_idx + 1] = (double)pi.y + MY * iv;
            A.cen[3 * out_idx + 2] = (double)pi.z + MZ * iv;
        }
        if (A.m2) A.m2[out_idx] = M2;
    }
    if (!A.rec) return;
    // neighbour threshold (in float32 in the FP32 form: the FP64 pipe is scarce)
    Real tau;
    if (Tol<Real>::fp32) {
        const float cv = cbrtf((float)V);
        tau = (Real)((float)Tol<Real>::area_rel * cv * cv);
    } else {
        tau = (Real)(Tol<Real>::area_rel * cbrt(V * V));
    }
    uint8_t* rec = A.rec + (size_t)out_idx * A.rec_stride;
    const bool geom = (A.emit & VT_EMIT_GEOM) != 0;
    int32_t* rfn = reinterpret_cast<int32_t*>(rec + REC_FNBR_OFF);
    uint8_t* rdeg = rec + REC_FDEG_OFF;
    uint8_t* rfv = rec + REC_FVTX_OFF;
    // One walk per face (a lane per plane) from its lowest live slot, so that
    // the sums and the emitted loops do not depend on thread timing: its area
    // (the neighbour test) and, with geometry, its loop of vertex ranks, at
    // the face's place in the record (an exclusive scan of (1, degree) over
    // the planes, T planes at a time)
    constexpr bool per = PER;
    int base_fi = 0, base_pos = 0;
    for (int f0 = 0; f0 < np; f0 += T) {
        const int f = f0 + gl;
        const int deg = f < np ? sm.u.tail.deg[f] : 0;
        int fi = 0, pos = 0;
        if (geom) {
            const int v = deg | ((deg ? 1 : 0) << 16);
            int inc = v;
#pragma unroll
            for (int d = 1; d < T; d <<= 1) {
                const int u = __shfl_up_sync(gmask, inc, d, T);
                if (gl >= d) inc += u;
            }
            const int tot = __shfl_sync(gmask, inc, T - 1, T);
            const int ex = inc - v;
            fi = base_fi + (ex >> 16);
            pos = base_pos + (ex & 0xffff);
            base_fi += tot >> 16;
            base_pos += tot & 0xffff;
        }
        if (f >= np) continue;
        const int src = sm.psrc[f];
        int oid = src;  // wall ids stay
        if (per) {  // the generator whose image the face faces; the cube's faces face the cell's own
            if (src < 0)
                oid = (int)out_idx;
            else if (deg > 0)
                oid = A.index_space == VT_INDEX_ORIGINAL ? __float_as_int(A.sorted[src & IMG_INDEX_MASK].w)
                                                         : (src & IMG_INDEX_MASK);
        } else if (src >= 0 && deg > 0 && A.index_space == VT_INDEX_ORIGINAL) {
            oid = __float_as_int(A.sorted[src].w);
        }
        Real area = 0;
        if (deg > 0) {
            const bool put = geom && fi < REC_FACES && pos + deg <= 3 * REC_VERTS;
            if (put) {
                rfn[fi] = oid;
                rdeg[fi] = (uint8_t)deg;
            }
            const Real fnx = sm.pnx[f], fny = sm.pny[f], fnz = sm.pnz[f];
            const Real sc = sm.u.tail.sc[f];
            const V4<Real> q = {fnx * sc, fny * sc, fnz * sc, (Real)0.5 / sqrt(fnx * fnx + fny * fny + fnz * fnz)};
            int cur = sm.u.tail.first[f];
            V4<Real> vc = ldv(sm.vpos, cur);
            for (int t2 = 0; t2 < deg; ++t2) {
                const uint32_t ids = *reinterpret_cast<const uint32_t*>(sm.vid[cur]);
                const uint32_t adj = *reinterpret_cast<const uint32_t*>(sm.vadj[cur]);
                const int t = ((ids & 0xff) == (uint32_t)f) ? 0 : ((((ids >> 8) & 0xff) == (uint32_t)f) ? 1 : 2);
                const int nxt = vt_ck((adj >> (8 * (t == 0 ? 2 : t - 1))) & 0xff, VCAP, CK_SLOT, A.st);
                const V4<Real> vn = ldv(sm.vpos, nxt);
                const Real ux = vc.x - q.x, uy = vc.y - q.y, uz = vc.z - q.z;
                const Real wx = vn.x - q.x, wy = vn.y - q.y, wz = vn.z - q.z;
                area += (uy * wz - uz * wy) * fnx + (uz * wx - ux * wz) * fny + (ux * wy - uy * wx) * fnz;
                if (put) rfv[vt_ck(pos + t2, 3 * REC_VERTS, CK_RECORD, A.st)] = (uint8_t)alive.rank(cur);
                cur = nxt;
                vc = vn;
            }
            area *= q.w;
        }
        // periodic: ids may repeat (two images of one generator); the key
        // id * PCAP + plane is unique and sorts the same (ids <= 2^24 - 2 and
        // planes < PCAP <= 128 keep it below the INT_MAX sentinel)
        const int key = per ? oid * PCAP + f : oid;
        put_key(sm.u.tail.sc, f, ((src >= 0 || per) && deg > 0 && area > tau) ? key : INT_MAX);
    }
    __syncwarp(gmask);
    // neighbours ascending: each key's rank among the keys
    int32_t* rnbr = reinterpret_cast<int32_t*>(rec + REC_NBR_OFF);
    int c = 0;
    for (int f = gl; f < np; f += T) {
        const int key = get_key(sm.u.tail.sc, f);
        if (key == INT_MAX) continue;
        ++c;
        int rank = 0;
        for (int g2 = 0; g2 < np; ++g2) rank += get_key(sm.u.tail.sc, g2) < key ? 1 : 0;
        if (rank < REC_FACES) rnbr[rank] = PER ? key / PCAP : key;
    }
    int nn_total = c;
#pragma unroll
    for (int o = T / 2; o >= 1; o >>= 1) nn_total += __shfl_xor_sync(gmask, nn_total, o, T);
    int nvtx = 0;
    if (geom) {
        nvtx = alive.count();
        double* rv = reinterpret_cast<double*>(rec + REC_VTX_OFF);
        float* rv32 = reinterpret_cast<float*>(rec + REC_VTX_OFF);
        for (int s = gl; s < VCAP; s += T) {
            if (!alive.test(s)) continue;
            const int li = alive.rank(s);
            if (li < REC_VERTS) {
                const V4<Real> v = ldv(sm.vpos, s);
                if (A.rec_f32) {  // half the record traffic; emit adds the generator in FP64
                    rv32[3 * li] = (float)v.x;
                    rv32[3 * li + 1] = (float)v.y;
                    rv32[3 * li + 2] = (float)v.z;
                } else {
                    rv[3 * li] = (double)pi.x + (double)v.x;
                    rv[3 * li + 1] = (double)pi.y + (double)v.y;
                    rv[3 * li + 2] = (double)pi.z + (double)v.z;
                }
            }
        }
    }
    if (gl == 0) {
        const int nface = geom ? base_fi : 0, nfv = geom ? base_pos : 0;
        const bool over = nn_total > REC_FACES || nface > REC_FACES || nvtx > REC_VERTS || nfv > 3 * REC_VERTS;
        if (over) atomicAdd((int*)&A.st->record_overflow, 1);
        RecHeader* hd = reinterpret_cast<RecHeader*>(rec);
        hd->nnbr = over ? 0 : nn_total;
        hd->nface = over ? 0 : nface;
        hd->nvtx = over ? 0 : nvtx;
        hd->nfv = over ? 0 : nfv;
        hd->p[0] = pi.x;
        hd->p[1] = pi.y;
        hd->p[2] = pi.z;
    }
    __syncwarp(gmask);
}

// NB batches of T candidates (sorted points of one shell) for the exhaustive
// walk; lane l holds candidates l, T + l, ... A generator q can cut the cell
// only if 4 R^2 > |q - p|^2 and its bisector n.x <= b (n = q - p,
// b = |n|^2 / 2) reaches beyond the cell's bounding box
// (sum_i max(n_i lo_i, n_i hi_i) > b); both tests run on every lane in float
// with margins that only admit extra candidates, and the survivors are clipped
// one at a time. Generators a resumed list already processed are skipped.
// RETEST: after each cut, the batch's other candidates are tested again
// against the smaller cell and the bounding box is refreshed; otherwise the
// box is refreshed once after the batch (a larger box only admits more
// candidates) and each candidate meets clip()'s own sign test. Measured on
// 1M points: the re-test pays in the FP32 walk of resumed cells (last pass
// 6.66 against 6.70 ms); without it the walk from the box is 8% faster
// (fused schedule 33.5 against 36.2 ms) and the FP64 walks 3-9%.
template <typename Real, int T, int VPL, int PCAP, bool PER, int NB, bool RETEST>
__device__ __forceinline__ int exhaustive_batch(Cell<Real, T, VPL, PCAP, PER>& cell, const Group<T>& G,
                                                typename Cell<Real, T, VPL, PCAP, PER>::S& sm, const ClipArgs& A,
                                                const GridDesc& grid, const bool (&valid)[NB], const int (&jj)[NB],
                                                const int (&code)[NB], double last_d2, int last_orig, float* lo3,
                                                float* hi3)
{
#ifdef VT_PROFILE
    const long long tb0 = clock64();
#endif
    const float4 pq = cell.pi;
    float px[NB], py[NB], pz[NB], ex[NB], ey[NB], ez[NB];
    uint32_t dkey[NB];
    unsigned mm[NB];
    unsigned any = 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        px[b] = py[b] = pz[b] = ex[b] = ey[b] = ez[b] = 0.f;
        bool need = false;
        if (valid[b]) {
            const float4 pc = A.sorted[img_index_t<PER>(jj[b])];
            px[b] = pc.x;
            py[b] = pc.y;
            pz[b] = pc.z;
            const float3 o = img_off_t<PER>(pq, pc, code[b], grid);
            ex[b] = o.x;
            ey[b] = o.y;
            ez[b] = o.z;
            const float d2 = fmaf(o.z, o.z, fmaf(o.y, o.y, o.x * o.x));
            const float r4 = 4.0f * (float)cell.R2;
            const float hb = fmaxf(o.x * lo3[0], o.x * hi3[0]) + fmaxf(o.y * lo3[1], o.y * hi3[1]) +
                             fmaxf(o.z * lo3[2], o.z * hi3[2]);
            need = r4 * (1.0f + 1e-4f) > d2 &&
                   hb > 0.5f * d2 * (1.0f - 1e-4f) - 1e-6f * sqrtf(d2 * (float)cell.R2) - 1e-30f &&
                   cell.reaches(sm, o.x, o.y, o.z);
            if (need && last_orig >= 0) {  // already processed from the list?
                const int ko = img_tie_t<PER>(pc, code[b]);
                if (Tol<Real>::fp32) {  // float keys compare in float (last_d2 holds a float)
                    const float kd = d2, ld = (float)last_d2;
                    if (kd < ld || (kd == ld && ko <= last_orig)) need = false;
                } else {
                    const double kd = img_key64(pq, A.sorted, jj[b], grid);
                    if (kd < last_d2 || (kd == last_d2 && ko <= last_orig)) need = false;
                }
            }
        }
        dkey[b] = __float_as_uint(fmaf(ez[b], ez[b], fmaf(ey[b], ey[b], ex[b] * ex[b])));
        mm[b] = G.ballot(need);
        any |= mm[b];
    }
#ifdef VT_PROFILE
    if (G.gl == 0) {
        int cnt = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) cnt += __popc(mm[b]);
        VT_PROF_ADD(8 + 7, cnt);
    }
    if (G.gl == 0) VT_PROF_ADD(21, clock64() - tb0);
    if (G.gl == 0 && any == 0) VT_PROF_ADD(23, 1);
    const long long tb1 = clock64();
#endif
    // survivors nearest first over all NB batches: the nearest cut most, so
    // the intermediate polyhedra stay small and fewer of the others still cut
    bool cut = false;
    while (any) {
        uint32_t mine = 0xffffffffu;  // this lane's nearest survivor (keys of finite d2 are smaller)
        int bs = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (((mm[b] >> G.gl) & 1u) && dkey[b] < mine) {
                mine = dkey[b];
                bs = b;
            }
        const uint32_t mn = __reduce_min_sync(G.mask, mine);
        const int src = __ffs(G.ballot(mine == mn)) - 1;
        const int bsrc = G.bcast(bs, src);
        float sx = px[0], sy = py[0], sz = pz[0];
        int sj = jj[0];
#pragma unroll
        for (int b = 1; b < NB; ++b)
            if (bs == b) {
                sx = px[b];
                sy = py[b];
                sz = pz[b];
                sj = jj[b];
            }
        any = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b == bsrc) mm[b] &= ~(1u << src);
            any |= mm[b];
        }
        float4 p;
        p.x = G.bcast(sx, src);
        p.y = G.bcast(sy, src);
        p.z = G.bcast(sz, src);
        p.w = 0.f;
        const int j = G.bcast(sj, src);
        // re-test against the current (smaller) cell
        const float3 o = img_off_t<PER>(pq, p, img_code_t<PER>(j), grid);
        const float d2 = fmaf(o.z, o.z, fmaf(o.y, o.y, o.x * o.x));
        const float hb =
            fmaxf(o.x * lo3[0], o.x * hi3[0]) + fmaxf(o.y * lo3[1], o.y * hi3[1]) + fmaxf(o.z * lo3[2], o.z * hi3[2]);
        if (!(4.0f * (float)cell.R2 * (1.0f + 1e-4f) > d2 &&
              hb > 0.5f * d2 * (1.0f - 1e-4f) - 1e-6f * sqrtf(d2 * (float)cell.R2) - 1e-30f))
            continue;
#ifdef VT_PROFILE
        const long long t0 = clock64();
#endif
        const int r = cell.clip_point(G, sm, p, j, A.sorted, grid, A.st);
#ifdef VT_PROFILE
        if (G.gl == 0) {
            VT_PROF_ADD(8 + 3, clock64() - t0);
            VT_PROF_ADD(8 + 4, 1);
            if (r == CLIP_CUT) VT_PROF_ADD(8 + 5, 1);
        }
#endif
        if (r == CLIP_OVERFLOW) return END_OVERFLOW;
        if (r == CLIP_INCONSISTENT) return END_INCONSISTENT;
        if (r == CLIP_CUT) {
            cut = true;
            if (RETEST) {
                // the box and the other survivors against the smaller cell
                cell.bbox(G, sm, lo3, hi3);
                any = 0;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (mm[b]) mm[b] &= G.ballot(((mm[b] >> G.gl) & 1u) && cell.reaches(sm, ex[b], ey[b], ez[b]));
                    any |= mm[b];
                }
            }
        }
    }
    if (!RETEST && cut) cell.bbox(G, sm, lo3, hi3);
#ifdef VT_PROFILE
    if (G.gl == 0) VT_PROF_ADD(22, clock64() - tb1);
#endif
    return 0;
}

// ---------------------------------------------------------------------------
// kernels: list mode (k > 0) and exhaustive mode (k == 0)
// ---------------------------------------------------------------------------
constexpr int CLIP_BLOCK = 128;
// resident blocks per SM the register budget aims for: the FP32 regular
// variants trade some spills for occupancy. The kernels that start every
// cell from the box (the list pass) run best at 7 blocks (72 registers), the
// ones that resume saved polyhedra (range lists) at 9 (56 registers):
// measured on the mixed cloud, list pass 11.67 / 11.84 / 11.91 ms and last
// pass 6.93 / 6.74 / 6.66 ms at 7 / 8 / 9 blocks. FP64 and robust keep 128
// registers
#ifndef VT_CLIP_MINB_F32
#define VT_CLIP_MINB_F32 7
#endif
#ifndef VT_CLIP_MINB_F32_RES
#define VT_CLIP_MINB_F32_RES 9
#endif
#ifndef VT_CLIP_MINB_F64
#define VT_CLIP_MINB_F64 4
#endif
// the FP32 walk kernel (latency-bound candidate batches): 6 blocks (measured
// against 4, 5, 7 and 8: the last pass 0.1-0.6 ms faster per 1M cells)
#ifndef VT_CLIP_MINB_EXH
#define VT_CLIP_MINB_EXH 6
#endif
// candidates per lane in one step of a walk from the box (fused schedule).
// Measured on 1M points: 1 is fastest (uniform 25.3 ms, clumps 35.2 ms of
// clipping), 2, 3 and 4 cost 20-70% more: every cut re-tests the remaining
// candidates of all NB batches against the whole polyhedron
#ifndef VT_WALK_NB
#define VT_WALK_NB 1
#endif
template <typename Real, bool ROBUST, bool EXH, bool RES>
constexpr int clip_minb()
{
    return (sizeof(Real) == 4 && !ROBUST)
               ? (EXH ? VT_CLIP_MINB_EXH : (RES ? VT_CLIP_MINB_F32_RES : VT_CLIP_MINB_F32))
               : VT_CLIP_MINB_F64;
}

// RES: the cells resume saved polyhedra (range lists, resumed lists, the
// walk); the kernels that start every cell from the box leave the resume
// code out (fewer live registers in their list loop)
template <typename Real, int T, int VPL, int PCAP, bool ROBUST, bool EXH, bool PER, bool RES>
__global__ void __launch_bounds__(CLIP_BLOCK, (clip_minb<Real, ROBUST, EXH, RES>())) k_clip(const __grid_constant__ ClipArgs A)
{
    using C = Cell<Real, T, VPL, PCAP, PER>;
    using S = typename C::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Group<T> G;
    S& sm = reinterpret_cast<S*>(smem_raw)[threadIdx.x / T];
    const int k = A.k;
    constexpr bool resume = RES && !ROBUST;
    // the robust exhaustive variant first clips by a nearest-first list, so
    // that its walk meets an almost final cell (the regular one resumes the
    // saved polyhedron of the last list pass instead)
    constexpr bool LIST = !EXH || ROBUST;
    // candidates per lane in one step of the walk (VT_WALK_NB batches of T
    // for a walk from the box, one batch for a resumed walk)
    constexpr int WNB = (!RES && !ROBUST) ? VT_WALK_NB : 1;
    int nq = (int)A.nq;
    if (A.nq_dev) {  // device-counted: list entries [nq_off, nq_off + nq_cap)
        const int64_t want = (int64_t)*A.nq_dev - A.nq_off;
        nq = (int)(want < 0 ? 0 : (want < A.nq_cap ? want : A.nq_cap));
    }
    C cell;
    cell.stamp = 0;
    // walks finished and generators they examined, added once per group
    unsigned walk_cells = 0, walk_cands = 0;

    // Cells come from a launch-wide counter, one per group at a time (cells
    // differ in cost by orders of magnitude: a static share per group leaves
    // the slowest groups running alone at the end). Cell indices fit 32 bits
    // (n < 2^30).
    auto next_cell = [&]() {
        int v = 0;
        if (G.gl == 0) v = atomicAdd(A.queue, 1);
        return G.bcast(v, 0);
    };
    for (int c = next_cell(); c < nq; c = next_cell()) {
        // this cell's list length; with k_next the doubled list follows at once:
        // validation is tested before every entry, so a cell that the first k
        // entries validate stops at entry k exactly as a re-queue would
        const int kc = A.klen ? A.klen[c] : (A.k_next > k ? A.k_next : k);
        if (kc < 0) continue;                    // no list: the cell is handled elsewhere
        const int q = A.queries ? A.queries[c] : (int)c;
        const GridDesc& grid = grid_of(A.g, A.sets, A.set_of, q);
        cell.pi = A.sorted[q];
        double last_d2 = -1.0;
        int last_orig = -1;
#ifdef VT_PROFILE
        long long tp0 = clock64();
        const int pb = EXH ? 8 : (A.complete ? 24 : 0);
#endif
        if (resume) {
            // the walk resumes from the last list key; list passes set it anew
            double ld;
            int lo;
            cell.restore(G, sm, A.state + (size_t)q * A.state_stride, ld, lo, A.sorted, grid);
            if (EXH) {
                last_d2 = ld;
                last_orig = lo;
            }
        }
        else cell.init_box(G, sm, grid);
        G.sync();
#ifdef VT_PROFILE
        long long tp1 = clock64();
        if (G.gl == 0) {
            VT_PROF_ADD(pb + 0, 1);
            VT_PROF_ADD(pb + 1, tp1 - tp0);
        }
#endif
        int end = END_NEED_K;
        if (LIST && k > 0) {
            // neighbour list, nearest first, from the first unprocessed entry;
            // each lane holds one entry of the current chunk of T (most lists
            // are one chunk: no prefetch, which would hold registers the
            // clipper needs)
            const int64_t li = (A.by_cell ? (int64_t)q : c) * (A.kstride ? A.kstride : k);
            const int32_t* nb = A.nbr + li;
            const Real* dd = reinterpret_cast<const Real*>(A.d2) + li;
            const int m0 = (resume && !A.restore) ? A.k_prev : 0;
            // From list entry kf on, only the entries whose bisector still
            // reaches the polyhedron are clipped: each lane tests its entry
            // against the live vertices once (at entry kf, or at the start of a
            // later chunk). A plane that misses the cell cannot cut the smaller
            // cells that follow, so skipping it changes no cell. kf: the second
            // half of a merged list (the first half starts from the box, where
            // every plane reaches), the whole of a resumed list.
            const int kf = A.complete ? m0 : (A.k_next > k ? k : (resume ? m0 : INT_MAX));
            bool stop = false;
            for (int base = m0; base < kc && !stop; base += T) {
                const int cj = base + G.gl < kc ? nb[base + G.gl] : -1;
                const Real cd = base + G.gl < kc ? dd[base + G.gl] : (Real)0;
                const float4 cp = cj >= 0 ? A.sorted[img_index_t<PER>(cj)] : make_float4(0.f, 0.f, 0.f, 0.f);
                const int cnt = kc - base < T ? kc - base : T;
                // range lists: each lane tests its entry against the live vertices
                // and only the entries that can cut are clipped, in list order
                // (in k-nearest lists most entries cut, so every one is clipped)
                const bool filtered = base >= kf;  // this whole chunk is tested at its start
                bool want = false;
                if (G.gl < cnt) {
                    if (!filtered || cj < 0) {
                        want = true;
                    } else {
                        const float3 o = img_off_t<PER>(cell.pi, cp, img_code_t<PER>(cj), grid);
                        want = cell.reaches(sm, o.x, o.y, o.z);
                    }
                }
                unsigned todo = G.ballot(want);
                bool tested = filtered;
                // cells still open at entry k of a merged list (a filtered chunk
                // may skip entry k itself: it is counted at the chunk's start)
                if (A.k_next > k && filtered && base == k && G.gl == 0) atomicAdd((int*)&A.st->n_second, 1);
                while (todo) {
                    const int t = __ffs(todo) - 1;
                    todo &= todo - 1u;
                    if (A.k_next > k && !filtered && base + t == k && G.gl == 0) atomicAdd((int*)&A.st->n_second, 1);
                    const int j = G.bcast(cj, t);
                    if (j < 0) { end = END_VALID; stop = true; break; }  // the list holds every other generator
                    const Real dj = G.bcast(cd, t);
                    if (cell.radius_ok(G, sm, dj, j, A.sorted, grid, A.st)) { end = END_VALID; stop = true; break; }
                    if (!tested && base + t >= kf) {
                        // entry kf inside this chunk: test it and the entries after it
                        bool reach = false;
                        if (G.gl >= t && G.gl < cnt) {
                            if (cj < 0) {
                                reach = true;
                            } else {
                                const float3 o = img_off_t<PER>(cell.pi, cp, img_code_t<PER>(cj), grid);
                                reach = cell.reaches(sm, o.x, o.y, o.z);
                            }
                        }
                        const unsigned rm = G.ballot(reach);
                        todo &= rm;
                        tested = true;
                        if (!((rm >> t) & 1u)) continue;  // entry t misses the cell
                    }
                    float4 p;
                    p.x = G.bcast(cp.x, t);
                    p.y = G.bcast(cp.y, t);
                    p.z = G.bcast(cp.z, t);
                    p.w = 0.f;
#ifdef VT_PROFILE
                    const long long t0 = clock64();
#endif
                    const int r = cell.clip_point(G, sm, p, j, A.sorted, grid, A.st);
#ifdef VT_PROFILE
                    if (G.gl == 0) {
                        VT_PROF_ADD(pb + 3, clock64() - t0);
                        VT_PROF_ADD(pb + 4, 1);
                        if (r == CLIP_CUT) VT_PROF_ADD(pb + 5, 1);
                    }
#endif
                    if (r == CLIP_OVERFLOW) { end = END_OVERFLOW; stop = true; break; }
                    if (r == CLIP_INCONSISTENT) { end = END_INCONSISTENT; stop = true; break; }
                }
            }
            if (!stop) {
                // a complete list leaves nothing that can cut; otherwise the
                // last entry bounds every generator the list does not hold
                if (A.complete) end = END_VALID;
                else if (kc > 0 && cell.radius_ok(G, sm, dd[kc - 1], nb[kc - 1], A.sorted, grid, A.st))
                    end = END_VALID;
            }
            if (end == END_NEED_K && kc > 0) {
                last_d2 = (double)dd[kc - 1];
                const int jl = nb[kc - 1];
                last_orig = img_tie_t<PER>(A.sorted[img_index_t<PER>(jl)], img_code_t<PER>(jl));
            }
        }
        if (EXH && end == END_NEED_K) {
            // exhaustive: every generator closer than 2R, by a shell walk
            const float4 pq = cell.pi;
            const int Gr = grid.G;
            const int32_t* coff = A.cell_off + grid.cell_base;
            const int ix = cell_coord(pq.x, grid.lo[0], grid.scale[0], Gr);
            const int iy = cell_coord(pq.y, grid.lo[1], grid.scale[1], Gr);
            const int iz = cell_coord(pq.z, grid.lo[2], grid.scale[2], Gr);
            float lo3[3], hi3[3];
            cell.bbox(G, sm, lo3, hi3);
            const float r_in2 = last_orig >= 0 ? (float)last_d2 * (1.0f - 1e-4f) : -1.0f;
            int status = 0;
            constexpr bool per = PER;
            for (int s = 0; status == 0; ++s) {
                // the shell's segments, T at a time, candidates spread over the lanes
                const bool wrap = per && (ix - s < 0 || iy - s < 0 || iz - s < 0 || ix + s >= Gr || iy + s >= Gr ||
                                          iz + s >= Gr);
                const int M = wrap ? seg_per_row(grid, s) : 2;
                const int nseg = M * (2 * s + 1) * (2 * s + 1);
#ifdef VT_PROFILE
                if (G.gl == 0) VT_PROF_ADD(16, 1);
#endif
                for (int e0 = 0; e0 < nseg && status == 0; e0 += T) {
#ifdef VT_PROFILE
                    if (G.gl == 0) VT_PROF_ADD(17, 1);
#endif
#ifdef VT_PROFILE
                    const long long ts0 = clock64();
#endif
                    // only grid cells that reach into the ball of radius 2R and are
                    // not wholly inside the ball the list already covered
                    int sa = 0, sb = 0, sc = IMG_NONE;
                    const float r_out2 = 4.0f * (float)cell.R2 * (1.0f + 2e-4f);
                    if (e0 + G.gl < nseg) {
                        if (wrap)
                            shell_segment_ball_p(e0 + G.gl, s, M, ix, iy, iz, grid, coff, pq, r_out2, r_in2, sa, sb,
                                                 sc);
                        else
                            shell_segment_ball(e0 + G.gl, s, ix, iy, iz, grid, coff, pq, r_out2, r_in2, sa, sb);
                    }
                    const int len = sb - sa;
                    int total;
                    const int start = G.scan(len, total);
                    walk_cands += (unsigned)total;
                    const int incl = start + len;
#ifdef VT_PROFILE
                    if (G.gl == 0) VT_PROF_ADD(19, total);
                    if (G.gl == 0) VT_PROF_ADD(20, clock64() - ts0);
#endif
                    for (int c0 = 0; c0 < total && status == 0; c0 += WNB * T) {
#ifdef VT_PROFILE
                        if (G.gl == 0) VT_PROF_ADD(18, 1);
#endif
                        bool vb[WNB];
                        int jb[WNB], cb[WNB];
#pragma unroll
                        for (int b = 0; b < WNB; ++b) {
                            const int i = c0 + b * T + G.gl;
                            int seg = 0;  // segments ending at or before i
#pragma unroll
                            for (int step = T / 2; step >= 1; step >>= 1)
                                if (G.bcast(incl, (seg + step - 1) & (T - 1)) <= i) seg += step;
                            const int aj = G.bcast(sa, seg & (T - 1)), sj = G.bcast(start, seg & (T - 1));
                            const int code = per ? G.bcast(sc, seg & (T - 1)) : IMG_NONE;
                            const int j0 = aj + (i - sj);
                            vb[b] = i < total && j0 != q;
                            jb[b] = per ? img_pack(j0, code) : j0;
                            cb[b] = code;
                        }
                        // (the robust variants keep the re-test: their slots are the last ones)
                        status = exhaustive_batch<Real, T, VPL, PCAP, PER, WNB,
                                                  ROBUST || (RES && sizeof(Real) == 4)>(
                            cell, G, sm, A, grid, vb, jb, cb, last_d2, last_orig, lo3, hi3);
                    }
                }
                if (status) break;
                if (per) {  // R <= |L| / 2: the walk ends within |L|
                    const float gap = shell_gap_p(grid, pq, ix, iy, iz, s);
                    if (gap > 0.0f && 4.0f * (float)cell.R2 * (1.0f + 2e-5f) <= gap * gap) { status = -1; break; }
                    continue;
                }
                const bool covers = ix - s <= 0 && iy - s <= 0 && iz - s <= 0 && ix + s >= Gr - 1 &&
                                    iy + s >= Gr - 1 && iz + s >= Gr - 1;
                if (covers) { status = -1; break; }
                const float gap = shell_gap(grid, pq, ix, iy, iz, s);
                if (gap > 0.0f && 4.0f * (float)cell.R2 * (1.0f + 2e-5f) <= gap * gap) { status = -1; break; }
            }
            end = status == -1 ? END_VALID : status;
            ++walk_cells;
        }

#ifdef VT_PROFILE
        long long tp2 = clock64();
        if (G.gl == 0) VT_PROF_ADD(pb + 2, tp2 - tp1);
#endif
        if (end == END_VALID) {
            G.sync();
            const int64_t out_idx = A.index_space == VT_INDEX_ORIGINAL ? (int64_t)__float_as_int(cell.pi.w) : (int64_t)q;
            finish_cell<Real, T, T * VPL, PCAP, typename C::M, PER>(sm, cell.alive, cell.np, cell.pi, G.gl, G.mask, out_idx,
                                                               A);
#ifdef VT_PROFILE
            if (G.gl == 0) VT_PROF_ADD(pb + 6, clock64() - tp2);
#endif
        } else {
            if (end == END_NEED_K && !EXH && !ROBUST && A.state)
                cell.save(G, sm, A.state + (size_t)q * A.state_stride, last_d2, last_orig);
            const int64_t out_idx = A.index_space == VT_INDEX_ORIGINAL ? (int64_t)__float_as_int(cell.pi.w) : (int64_t)q;
            if (G.gl == 0) {
                if (A.rec) {
                    RecHeader* hd = reinterpret_cast<RecHeader*>(A.rec + (size_t)out_idx * A.rec_stride);
                    hd->nnbr = hd->nface = hd->nvtx = hd->nfv = 0;
                }
                if (end == END_NEED_K && !EXH) {
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
    if (EXH && G.gl == 0 && walk_cells) {
        atomicAdd(&A.st->walk_cells, (unsigned long long)walk_cells);
        atomicAdd(&A.st->walk_cands, (unsigned long long)walk_cands);
    }
}

template <typename Real, int T, int VPL, int PCAP>
constexpr size_t state_bytes()
{
    return StateLayout<Real, T * VPL, PCAP>::BYTES;
}

template <typename Real, int T, int VPL, int PCAP, bool ROBUST>
cudaError_t launch_variant(const ClipArgs& a, cudaStream_t s)
{
    using S = GroupSmem<Real, T * VPL, PCAP>;
    const size_t smem = sizeof(S) * (CLIP_BLOCK / T);
    // periodic boxes have their own instantiations (the walls' kernels keep their registers)
    const bool res = !ROBUST && a.state && (a.k_prev > 0 || a.restore);
    auto kern = a.g.periodic
                    ? (a.exhaustive ? (res ? k_clip<Real, T, VPL, PCAP, ROBUST, true, true, true>
                                           : k_clip<Real, T, VPL, PCAP, ROBUST, true, true, false>)
                                    : (res ? k_clip<Real, T, VPL, PCAP, ROBUST, false, true, true>
                                           : k_clip<Real, T, VPL, PCAP, ROBUST, false, true, false>))
                    : (a.exhaustive ? (res ? k_clip<Real, T, VPL, PCAP, ROBUST, true, false, true>
                                           : k_clip<Real, T, VPL, PCAP, ROBUST, true, false, false>)
                                    : (res ? k_clip<Real, T, VPL, PCAP, ROBUST, false, false, true>
                                           : k_clip<Real, T, VPL, PCAP, ROBUST, false, false, false>));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // as many blocks as are resident at once (they take cells from the queue)
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CLIP_BLOCK, smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int gpb = CLIP_BLOCK / T;
    int64_t blocks = (a.nq + gpb - 1) / gpb;
    const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > resident) blocks = resident;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, CLIP_BLOCK, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

}  // namespace vt
