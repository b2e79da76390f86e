// Integer grid records of the tensor-core pre-test (TDQ_MODE_TC_FILTER).
//
// The pre-test asks, for every candidate (entry, query segment) pair, whether
// the bounding spheres of the two segments -- the entry's, and the query's
// grown by d -- can meet.  If they cannot, the two moving points are never
// within d of each other (Sec. 3: each point stays on its segment), so the
// pair is dropped; otherwise the FP64 path decides it (Sec. 5, Algorithm 1).
//
// Every sphere is snapped to an integer grid: center u = rint((c - o) lam)
// per axis, clamped to [-kTcC, kTcC], and radius rho, the smallest integer
// >= lam (r (1 + 2^-20) + 2^-40 (max|c| + r) + 2^-60) + sqrt(3)/2 + 2^-20.
// Rounding a center moves it by at most sqrt(3)/2 grid units; clamping a
// query center to the grid's box (which holds every entry center) does not
// increase its distance to any entry; the relative and absolute terms cover
// the FP64 rounding of the centers and radii and of the positions and the
// decision the FP64 path computes.  So
//     |u_e - u_q| <= rho_e + rho_q
// holds for every pair the FP64 path can accept.  In integers,
//     v = |u_e|^2 - rho_e^2 + |u_q|^2 - rho_q^2 - 1 - 2 u_e.u_q - 2 rho_e rho_q
// is negative exactly then.  v is the dot product of two 16-element records
//     entry  a = (ux, uy, uz, rho, A_hi, A_lo, 2048, 1, f, 0...)
//     query  b = (-2ux, -2uy, -2uz, -2rho, 2048, 1, B_hi, B_lo, 1, 0...)
// with A = |u_e|^2 - rho_e^2 = 2048 A_hi + A_lo, B = |u_q|^2 - rho_q^2 - 1 =
// 2048 B_hi + B_lo, 0 <= A_lo, B_lo < 2048, f = 0: a GEMM of the entries'
// records with the queries' (tcgen05.mma kind::f16, FP32 accumulation).
// Every element is an integer FP16 represents exactly (|x| <= 2048, or even
// and <= 4096), every product is exact in FP32, and with |u| <= 1023 and
// rho <= 1023 the sum of the magnitudes of all products is below 2^24, so
// every partial sum is an integer FP32 holds exactly: the MMA computes v
// without rounding, in any order.
//
// A sphere too large for the grid (rho > kTcP) gets a record that makes v
// negative against every partner: entry (0,...,0, f = -1), query (0,...,0,
// B_lo = -1, 1).  Such pairs always go on to the FP64 path.
#pragma once

#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

namespace tdq {

constexpr int kTcC = 1023;  // grid coordinates lie in [-kTcC, kTcC]
constexpr int kTcP = 1023;  // grid radii lie in [0, kTcP]

// The grid: origin o and scale lam (grid units per unit of length).
struct TcGrid {
    double ox, oy, oz, lam;
};

__host__ __device__ inline TcGrid tc_grid_from_box(double xmin, double xmax, double ymin, double ymax, double zmin,
                                                   double zmax)
{
    TcGrid g;
    g.ox = 0.5 * xmin + 0.5 * xmax;
    g.oy = 0.5 * ymin + 0.5 * ymax;
    g.oz = 0.5 * zmin + 0.5 * zmax;
    double ext = fmax(xmax - xmin, fmax(ymax - ymin, zmax - zmin));
    double lam = 2.0 * kTcC / ext;
    // empty extent: any scale (every center maps to 0); an extent too large
    // or too small for a finite scale gives lam = 0, which makes every
    // radius "too large" (every pair goes on to the FP64 path)
    g.lam = (ext > 0.0 && isfinite(lam)) ? lam : (ext > 0.0 ? 0.0 : 1.0);
    return g;
}

__device__ __forceinline__ int tc_coord(double c, double o, double lam)
{
    const double u = rint((c - o) * lam);
    return (int)fmin(fmax(u, -(double)kTcC), (double)kTcC);  // +-inf clamp; NaN never reaches here
}

// Grid radius of a sphere of radius r (>= 0) whose center's largest
// coordinate magnitude is m; -1 when it exceeds kTcP (or is not finite).
__device__ __forceinline__ int tc_radius(double r, double m, double lam)
{
    const double t = lam * (r * (1.0 + 0x1p-20) + 0x1p-40 * (m + r) + 0x1p-60) + 0.8660254037844387 + 0x1p-20;
    if (!(lam > 0.0) || !(t <= (double)kTcP)) return -1;
    return (int)ceil(t);
}

__device__ __forceinline__ uint32_t tc_pack(int lo, int hi)
{
    const __half a = __int2half_rn(lo), b = __int2half_rn(hi);
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// floor division of x by 2048 and the remainder in [0, 2048)
__device__ __forceinline__ void tc_split(int64_t x, int &hi, int &lo)
{
    const int64_t h = x >= 0 ? x / 2048 : -((-x + 2047) / 2048);
    hi = (int)h;
    lo = (int)(x - h * 2048);
}

// Entry record of the sphere (center c, radius r).
__device__ __forceinline__ void tc_entry_record(double cx, double cy, double cz, double r, const TcGrid &g,
                                                uint4 &lo, uint4 &hi)
{
    const double m = fmax(fabs(cx), fmax(fabs(cy), fabs(cz)));
    const int rho = tc_radius(r, m, g.lam);
    if (rho < 0) {
        lo = make_uint4(0u, 0u, 0u, 0u);
        hi = make_uint4(tc_pack(-1, 0), 0u, 0u, 0u);
        return;
    }
    const int x = tc_coord(cx, g.ox, g.lam), y = tc_coord(cy, g.oy, g.lam), z = tc_coord(cz, g.oz, g.lam);
    const int64_t A = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z - (int64_t)rho * rho;
    int ah, al;
    tc_split(A, ah, al);
    lo = make_uint4(tc_pack(x, y), tc_pack(z, rho), tc_pack(ah, al), tc_pack(2048, 1));
    hi = make_uint4(0u, 0u, 0u, 0u);
}

// Query record of the sphere (center c, radius r) grown by d.
__device__ __forceinline__ void tc_query_record(double cx, double cy, double cz, double r, double d,
                                                const TcGrid &g, uint4 &lo, uint4 &hi)
{
    const double m = fmax(fabs(cx), fmax(fabs(cy), fabs(cz)));
    const int rho = tc_radius(r + d, m, g.lam);
    if (rho < 0) {
        lo = make_uint4(0u, 0u, 0u, tc_pack(0, -1));
        hi = make_uint4(tc_pack(1, 0), 0u, 0u, 0u);
        return;
    }
    const int x = tc_coord(cx, g.ox, g.lam), y = tc_coord(cy, g.oy, g.lam), z = tc_coord(cz, g.oz, g.lam);
    const int64_t B = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z - (int64_t)rho * rho - 1;
    int bh, bl;
    tc_split(B, bh, bl);
    lo = make_uint4(tc_pack(-2 * x, -2 * y), tc_pack(-2 * z, -2 * rho), tc_pack(2048, 1), tc_pack(bh, bl));
    hi = make_uint4(tc_pack(1, 0), 0u, 0u, 0u);
}

// Records are stored in groups of 8 (the MMA's 8-row core matrices): record
// k's first 16 bytes at uint4 index (k / 8) * 16 + k % 8, its last 16 bytes
// 8 uint4 further.  128 consecutive records (k0 a multiple of 8) are then one
// contiguous 4 KB block in the no-swizzle K-major layout the MMA reads with
// core matrices 128 B apart along K and 256 B apart along M/N.
__device__ __forceinline__ void tc_store(uint4 *rec, uint64_t k, uint4 lo, uint4 hi)
{
    const uint64_t b = (k >> 3) * 16 + (k & 7);
    rec[b] = lo;
    rec[b + 8] = hi;
}

}  // namespace tdq
