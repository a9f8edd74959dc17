// tile.cuh -- the per-tile FP32 shooting routine (Algorithm 1 on one 64 x 8*NP
// tile of the ray grid: prologue, star stages, beta, binning), shared by the
// single-field kernel, the persistent multi-field kernel and the fallback tiles
// of the learned-far-field kernel.  See shoot_fp32.cu for the design notes.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "mlens_dev.cuh"

namespace mlens {

namespace cg = cooperative_groups;

constexpr int kThreads = 256;
constexpr int kTileX = 64;                 // rays per tile row = threads per row group
constexpr int kGroups = kThreads / kTileX; // row groups
constexpr int kKahan = 32;                 // stars per compensated partial

static_assert(kStarPad % kKahan == 0, "star padding must be whole Kahan chunks");

template <int SC>
struct StarStage {
    float4 q[2][SC];   // (-dx, -dx, -dy, -dy) relative to the tile centre
    float2 mm[2][SC];  // (m, m)
};

template <int SC>
union ShootSmem {
    StarStage<SC> st;
    uint32_t hist[kWin * kWin];
};

struct TileShared {
    float tc[10];      // cx, cy, ex, ey, B0h.x, B0h.y, B0l.x, B0l.y, exl, eyl
    int win[2];
    unsigned sred[3];
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// v - c for packed pairs, with one rounding (fma with -1 is exact in the product)
__device__ __forceinline__ float2 sub2(float2 v, float2 c) { return __ffma2_rn(c, f2(-1.0f, -1.0f), v); }

// The tile centre on one axis, chosen so that the offset of every star near the
// tile from it is exact in float32: 0 when the tile lies within 4 tile extents of
// the axis' zero (a star offset is then the star's own coordinate), else the
// middle of the tile rounded to a multiple of q, the largest power of two not
// above the ray spacing (RayGrid qx, qy).  A float star coordinate s and a centre
// c that are both multiples of ulp(s), or both of q, differ by a float whenever
// |s - c| < |s| (or |s - c| < 2^24 q), which holds for the stars within an extent
// of the tile (|s| >= 2.5 extents > |s - c|).  Farther stars round as before,
// with errors small against their distance.
__device__ __forceinline__ float tile_centre(double mid, double extent, double q, double qinv)
{
    if (fabs(mid) < 4.0 * extent) return 0.0f;
    const double c = rint(mid * qinv) * q;
    return (float)c == c ? (float)c : (float)mid;
}

// Offset of ray k of the tile from the tile centre, e + k d with the first ray's
// offset e = eh + el and the ray spacing d = dh + dl, as a float pair (hi, lo):
// TwoProduct for k dh (exact with the FMA), TwoSum with eh, the small terms
// added to the error and the pair renormalised; about 2^-44 relative.  The
// star loop adds lo after the subtraction of the star's offset, which is exact
// for the stars close to the ray (tile_centre): there the deflection m/r would
// magnify the rounding of a float32 offset.  On grids whose ray offsets are
// exact floats (a dyadic spacing and origin, RayGrid lo = 0) lo is zero and the
// loop skips the addition, which then changes nothing.
__device__ __forceinline__ void ray_offset(float k, float eh, float el, float dh, float dl, float &hi, float &lo)
{
    const float p = __fmul_rn(k, dh);
    const float pe = __fmaf_rn(k, dh, -p);
    const float s = __fadd_rn(eh, p);
    const float bb = __fsub_rn(s, eh);
    const float se = __fadd_rn(__fsub_rn(eh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    const float t = __fadd_rn(__fadd_rn(se, pe), __fmaf_rn(k, dl, el));
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// Kahan step on packed pairs: S + v with compensation C (true sum ~ S - C).
__device__ __forceinline__ void kahan2(float2 &S, float2 &C, float2 v)
{
    float2 y = sub2(v, C);
    float2 t = __fadd2_rn(S, y);
    C = sub2(sub2(t, S), y);
    S = t;
}

constexpr int tile_rows(int np) { return kGroups * 2 * np; }

// Reciprocal on the FMA pipe for a packed pair: an initial guess read off the
// float bits (seed - bits(x), seed chosen by a minimax search over one binade:
// relative error <= 5.1%) refined by three Newton-Raphson steps
// y <- y + y (1 - x y), each squaring the relative error (5.1e-2 -> 2.6e-3 ->
// 6.5e-6 -> 4e-11, below float32 resolution).  x = 0 gives a non-finite result,
// as the hardware reciprocal does.  Used for a share of the interactions so that
// the FMA pipe takes part of the reciprocal load off the MUFU unit.
constexpr int kRcpSeed = 0x7EF311C2;

__device__ __forceinline__ float2 rcp_nr2(float2 x)
{
    float2 y = f2(__int_as_float(kRcpSeed - __float_as_int(x.x)), __int_as_float(kRcpSeed - __float_as_int(x.y)));
    const float2 nx = f2(-x.x, -x.y);
    const float2 one = f2(1.0f, 1.0f);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float2 e = __ffma2_rn(nx, y, one);
        y = __ffma2_rn(y, e, y);
    }
    return y;
}

// One tile (bx, by) of the ray grid of `a`, start to finish: prologue, star
// stages, beta, binning, counters.  Every thread of the CTA must call it.
// NRP = 1: ray pair 0 takes its reciprocals from rcp_nr2 (FMA pipe) on every third
// star of a 32-star chunk (stars 2, 5, .., 29: 10 of the 128 reciprocals a thread
// forms per chunk, 7.8 %); all others come from the MUFU unit.  That share
// balances the two pipes best on GB300 (measured: 4.84e12 interactions/s against
// 4.67e12 with MUFU alone, 4.79e12 at 1/8 and 4.39e12 at 1/4 of the reciprocals).
// NRP = 0: MUFU alone.
//
// SPLIT > 1 (re-centred FP32 only): the CTA is rank r of a cluster of SPLIT CTAs
// that share the tile; it sums the r-th of SPLIT consecutive 32-aligned slices
// of the stars.  Ranks 1.. leave their (S, C) partials in `part` (2 NP float4
// per thread, in their own shared memory); rank 0 reads them through
// distributed shared memory in rank order, folds each in with two Kahan steps
// (S_r, then -C_r) and alone goes on to beta and binning.
// LOM: how the tile learns whether the ray offsets need low parts: 0 = from the grid
// at run time (RayGrid lo, both loops compiled), 1 = never, 2 = always (callers
// that have chosen already).
//
// GS (re-centred FP32 only, SPLIT = 1): the split star sum through global memory.
// GS = 1: the CTA sums slice `gslice` of a.gslices consecutive 32-aligned slices of
// the stars (the same slices as a cluster split of that many CTAs) and stores its
// partials (S, C) as 2 NP float4 per thread at a.gpart, block gtile * a.gslices +
// gslice, then returns.  GS = 2: the CTA sums no stars; it takes slice 0's partials
// as its own, folds the others in slice order (two Kahan steps each, S_r then -C_r,
// as the cluster fold does) and goes on to beta and binning.
template <int NP, int SC, bool NAIVE, int NRP = 0, int SPLIT = 1, int LOM = 0, int GS = 0>
__device__ __forceinline__ void shoot_tile(const ShootArgs &a, int bx, int by, ShootSmem<SC> &sm, TileShared &ts,
                                           float4 *part = nullptr, int64_t gtile = 0, int gslice = 0)
{
    static_assert(SPLIT == 1 || !NAIVE, "the split sum is for the re-centred kernel");
    static_assert(GS == 0 || (!NAIVE && SPLIT == 1), "the global split is for the re-centred kernel");
    constexpr int kTileY = tile_rows(NP);
    constexpr int kLoads = (SC + kThreads - 1) / kThreads;
    const int tid = threadIdx.x;
    const int tx = tid % kTileX;
    const int tg = tid / kTileX;
    const int i0 = bx * kTileX;
    const int j0 = by * kTileY;
    const RayGrid &R = a.rays;

    if (tid == 0) {
        if (!NAIVE) {
            // tile centre (tile_centre: star offsets near the tile exact), offsets of
            // the first ray and A c in FP64, split into float pairs
            double cxd = R.x0 + ((double)i0 + 0.5 * kTileX) * R.dx;
            double cyd = R.y0 + ((double)j0 + 0.5 * kTileY) * R.dy;
            float cx = tile_centre(cxd, kTileX * R.dx, R.qx, R.qxinv), cy = tile_centre(cyd, kTileY * R.dy, R.qy, R.qyinv);
            double ex = (R.x0 + ((double)i0 + 0.5) * R.dx) - (double)cx;
            double ey = (R.y0 + ((double)j0 + 0.5) * R.dy) - (double)cy;
            double bxd = a.lens.a11 * (double)cx + a.lens.a12 * (double)cy;
            double byd = a.lens.a12 * (double)cx + a.lens.a22 * (double)cy;
            float bxh = (float)bxd, byh = (float)byd;
            ts.tc[0] = cx;
            ts.tc[1] = cy;
            ts.tc[2] = (float)ex;
            ts.tc[3] = (float)ey;
            ts.tc[4] = bxh;
            ts.tc[5] = byh;
            ts.tc[6] = (float)(bxd - (double)bxh);
            ts.tc[7] = (float)(byd - (double)byh);
            ts.tc[8] = (float)(ex - (double)ts.tc[2]);
            ts.tc[9] = (float)(ey - (double)ts.tc[3]);
        }
        ts.sred[0] = ts.sred[1] = ts.sred[2] = 0u;
    }
    __syncthreads();

    // ------------------------------------------------------- this thread's rays
    float2 rx;       // packed (x, x): both rays of a pair share the column
    float2 ry[NP];   // packed (y_2p, y_2p+1)
    float2 rxl, ryl[NP];               // low parts of the offsets (re-centred variants)
    float2 px[NP], py[NP];             // partial sums (NAIVE: the whole running sum)
    float2 Sx[NP], Sy[NP], Cx[NP], Cy[NP];
    const float kx = (float)tx;
    float cx = 0.f, cy = 0.f;
    const bool lo = !NAIVE && (LOM == 2 || (LOM == 0 && R.lo));
    if (!NAIVE) {
        cx = ts.tc[0];
        cy = ts.tc[1];
        if (lo) {
            float h, l;
            ray_offset(kx, ts.tc[2], ts.tc[8], R.dxh, R.dxl, h, l);
            rx = f2(h, h);
            rxl = f2(l, l);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float k0 = (float)(tg * 2 * NP + 2 * p), k1 = k0 + 1.0f;
                float h1, l1;
                ray_offset(k0, ts.tc[3], ts.tc[9], R.dyh, R.dyl, h, l);
                ray_offset(k1, ts.tc[3], ts.tc[9], R.dyh, R.dyl, h1, l1);
                ry[p] = f2(h, h1);
                ryl[p] = f2(l, l1);
            }
        } else {
            // exact float offsets (RayGrid lo = 0): e + k d with every step exact
            const float dxr = __fmaf_rn(kx, R.dxh, ts.tc[2]);
            rx = f2(dxr, dxr);
            rxl = f2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float k0 = (float)(tg * 2 * NP + 2 * p), k1 = k0 + 1.0f;
                ry[p] = f2(__fmaf_rn(k0, R.dyh, ts.tc[3]), __fmaf_rn(k1, R.dyh, ts.tc[3]));
                ryl[p] = f2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) px[p] = py[p] = Sx[p] = Sy[p] = Cx[p] = Cy[p] = f2(0.f, 0.f);
    } else {
        const float x0f = (float)R.x0, y0f = (float)R.y0;
        const float dxf = (float)R.dx, dyf = (float)R.dy;
        float thx = x0f + ((float)(i0 + tx) + 0.5f) * dxf;
        rx = f2(thx, thx);
        rxl = f2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float y0 = y0f + ((float)(j0 + tg * 2 * NP + 2 * p) + 0.5f) * dyf;
            float y1 = y0f + ((float)(j0 + tg * 2 * NP + 2 * p + 1) + 0.5f) * dyf;
            ry[p] = f2(y0, y1);
            ryl[p] = f2(0.f, 0.f);
            // alpha_0 first (Algorithm 1), then every star is added to it
            px[p] = f2(a.lens.fm11 * thx + a.lens.fm12 * y0, a.lens.fm11 * thx + a.lens.fm12 * y1);
            py[p] = f2(a.lens.fm12 * thx + a.lens.fm22 * y0, a.lens.fm12 * thx + a.lens.fm22 * y1);
            Sx[p] = Sy[p] = Cx[p] = Cy[p] = f2(0.f, 0.f);
        }
    }

    // ---------------------------------------------------------- star stages
    const float4 *stars = a.stars;
    int64_t nst = a.nstars;  // multiple of kKahan
    if (SPLIT > 1) {
        const int64_t chunk = ((nst + SPLIT - 1) / SPLIT + kKahan - 1) / kKahan * kKahan;
        const int64_t s0 = min(nst, (int64_t)cg::this_cluster().block_rank() * chunk);
        stars += s0;
        nst = min(chunk, nst - s0);
    }
    if (GS == 1) {
        const int64_t chunk = ((nst + a.gslices - 1) / a.gslices + kKahan - 1) / kKahan * kKahan;
        const int64_t s0 = min(nst, (int64_t)gslice * chunk);
        stars += s0;
        nst = min(chunk, nst - s0);
    }
    if (GS == 2) nst = 0;
    const int nstage = (int)((nst + SC - 1) / SC);
    float4 nxt[kLoads];
    auto stage_load = [&](int s) {
        const int64_t base = (int64_t)s * SC;
#pragma unroll
        for (int l = 0; l < kLoads; ++l) {
            const int k = tid + l * kThreads;
            nxt[l] = (k < SC && base + k < nst) ? __ldg(&stars[base + k]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto stage_store = [&](int buf) {
#pragma unroll
        for (int l = 0; l < kLoads; ++l) {
            const int k = tid + l * kThreads;
            if (k < SC) {
                const float4 q = nxt[l];
                float nx = NAIVE ? -q.x : __fsub_rn(cx, q.x);
                float ny = NAIVE ? -q.y : __fsub_rn(cy, q.y);
                sm.st.q[buf][k] = make_float4(nx, nx, ny, ny);
                sm.st.mm[buf][k] = f2(q.z, q.z);
            }
        }
    };
    if (nstage > 0) {
        stage_load(0);
        stage_store(0);
    }
    __syncthreads();

    for (int s = 0; s < nstage; ++s) {
        const int buf = s & 1;
        const int cnt = (int)min((int64_t)SC, nst - (int64_t)s * SC);
        if (s + 1 < nstage) stage_load(s + 1);
        const float4 *Q = sm.st.q[buf];
        const float2 *M = sm.st.mm[buf];
        // the chunks of the stage; LO: the offsets' low parts are added after the
        // subtraction (grids whose ray offsets are not exact floats, RayGrid lo)
        auto chunks = [&](auto lo_tag) {
            constexpr bool LO = decltype(lo_tag)::value && !NAIVE;
#pragma unroll 1
            for (int k0 = 0; k0 < cnt; k0 += kKahan) {
#pragma unroll
                for (int k = k0; k < k0 + kKahan; ++k) {
                    const float4 q = Q[k];
                    const float2 m2 = M[k];
                    const float2 dx = LO ? __fadd2_rn(__fadd2_rn(rx, f2(q.x, q.y)), rxl) : __fadd2_rn(rx, f2(q.x, q.y));
                    const float2 dx2 = __fmul2_rn(dx, dx);
                    const float2 nyv = f2(q.z, q.w);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const float2 dy = LO ? __fadd2_rn(__fadd2_rn(ry[p], nyv), ryl[p]) : __fadd2_rn(ry[p], nyv);
                        const float2 r2 = __ffma2_rn(dy, dy, dx2);
                        const float2 inv = NRP > 0 && p == 0 && (k - k0) % 3 == 2 ? rcp_nr2(r2)
                                                                                 : f2(rcp_approx(r2.x), rcp_approx(r2.y));
                        const float2 f = __fmul2_rn(m2, inv);
                        px[p] = __ffma2_rn(f, dx, px[p]);
                        py[p] = __ffma2_rn(f, dy, py[p]);
                    }
                }
                if (!NAIVE) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        kahan2(Sx[p], Cx[p], px[p]);
                        kahan2(Sy[p], Cy[p], py[p]);
                        px[p] = py[p] = f2(0.f, 0.f);
                    }
                }
            }
        };
        if (LOM == 2 && !NAIVE)
            chunks(std::true_type{});
        else if (LOM == 1 || NAIVE)
            chunks(std::false_type{});
        else if (lo)
            chunks(std::true_type{});
        else
            chunks(std::false_type{});
        if (s + 1 < nstage) stage_store(buf ^ 1);
        __syncthreads();
    }

    if constexpr (GS == 1) {
        float4 *dst = a.gpart + (gtile * a.gslices + gslice) * (int64_t)(2 * NP * kThreads);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            dst[(2 * p) * kThreads + tid] = make_float4(Sx[p].x, Sx[p].y, Sy[p].x, Sy[p].y);
            dst[(2 * p + 1) * kThreads + tid] = make_float4(Cx[p].x, Cx[p].y, Cy[p].x, Cy[p].y);
        }
        return;
    }
    if constexpr (GS == 2) {
        const float4 *src = a.gpart + gtile * a.gslices * (int64_t)(2 * NP * kThreads);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const float4 s0 = src[(2 * p) * kThreads + tid], c0 = src[(2 * p + 1) * kThreads + tid];
            Sx[p] = f2(s0.x, s0.y);
            Sy[p] = f2(s0.z, s0.w);
            Cx[p] = f2(c0.x, c0.y);
            Cy[p] = f2(c0.z, c0.w);
        }
#pragma unroll 1
        for (int r = 1; r < a.gslices; ++r) {
            const float4 *rp = src + (int64_t)r * (2 * NP * kThreads);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float4 sr = rp[(2 * p) * kThreads + tid], cr = rp[(2 * p + 1) * kThreads + tid];
                kahan2(Sx[p], Cx[p], f2(sr.x, sr.y));
                kahan2(Sy[p], Cy[p], f2(sr.z, sr.w));
                kahan2(Sx[p], Cx[p], f2(-cr.x, -cr.y));
                kahan2(Sy[p], Cy[p], f2(-cr.z, -cr.w));
            }
        }
    }

    if constexpr (SPLIT > 1) {
        cg::cluster_group cl = cg::this_cluster();
        const unsigned rank = cl.block_rank();
        if (rank != 0) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                part[(2 * p) * kThreads + tid] = make_float4(Sx[p].x, Sx[p].y, Sy[p].x, Sy[p].y);
                part[(2 * p + 1) * kThreads + tid] = make_float4(Cx[p].x, Cx[p].y, Cy[p].x, Cy[p].y);
            }
        }
        cl.sync();  // every rank's partials are in place
        if (rank == 0) {
#pragma unroll 1
            for (int r = 1; r < SPLIT; ++r) {
                const float4 *rp = cl.map_shared_rank(part, r);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float4 sr = rp[(2 * p) * kThreads + tid], cr = rp[(2 * p + 1) * kThreads + tid];
                    kahan2(Sx[p], Cx[p], f2(sr.x, sr.y));
                    kahan2(Sy[p], Cy[p], f2(sr.z, sr.w));
                    kahan2(Sx[p], Cx[p], f2(-cr.x, -cr.y));
                    kahan2(Sy[p], Cy[p], f2(-cr.z, -cr.w));
                }
            }
        }
        cl.sync();  // rank 0 has read them: the other ranks may exit
        if (rank != 0) return;
    }

    // ------------------------------------------------ beta as float pairs
    float bxh[2 * NP], byh[2 * NP], bxl[2 * NP], byl[2 * NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = 2 * p + h;
            if (!NAIVE) {
                const float sx = h ? Sx[p].y : Sx[p].x, sy = h ? Sy[p].y : Sy[p].x;
                const float ccx = h ? Cx[p].y : Cx[p].x, ccy = h ? Cy[p].y : Cy[p].x;
                const float dxr = rx.x, dyr = h ? ry[p].y : ry[p].x;
                const float dxl = rxl.x, dyl = h ? ryl[p].y : ryl[p].x;
                // A delta for this ray (small), the offsets' low parts included
                const float lx = __fmaf_rn(a.lens.fa11, dxr, __fmaf_rn(a.lens.fa12, dyr,
                                           __fmaf_rn(a.lens.fa11, dxl, __fmul_rn(a.lens.fa12, dyl))));
                const float ly = __fmaf_rn(a.lens.fa12, dxr, __fmaf_rn(a.lens.fa22, dyr,
                                           __fmaf_rn(a.lens.fa12, dxl, __fmul_rn(a.lens.fa22, dyl))));
                float th, tl;
                two_sum(ts.tc[4], -sx, th, tl);
                tl = __fadd_rn(tl, __fadd_rn(__fadd_rn(ts.tc[6], ccx), lx));
                two_sum(th, tl, bxh[r], bxl[r]);
                two_sum(ts.tc[5], -sy, th, tl);
                tl = __fadd_rn(tl, __fadd_rn(__fadd_rn(ts.tc[7], ccy), ly));
                two_sum(th, tl, byh[r], byl[r]);
            } else {
                const float thy = h ? ry[p].y : ry[p].x;
                bxh[r] = __fsub_rn(rx.x, h ? px[p].y : px[p].x);
                byh[r] = __fsub_rn(thy, h ? py[p].y : py[p].x);
                bxl[r] = 0.0f;
                byl[r] = 0.0f;
            }
        }
    }

    // ----------------------------------------------------------- binning
    const int ix = i0 + tx;
    const bool col_ok = ix < R.nx;
    __syncthreads();  // star stages are dead: reuse the memory as the window
    hist_zero(sm.hist);
    if (tid == 0) {
        ts.win[0] = pair_axis_rough(bxh[0], a.bin.ax) - kWin / 2;
        ts.win[1] = pair_axis_rough(byh[0], a.bin.ay) - kWin / 2;
    }
    __syncthreads();
    WinHist W{sm.hist, ts.win[0], ts.win[1]};
    unsigned nb = 0, no = 0, nn = 0;
#pragma unroll
    for (int r = 0; r < 2 * NP; ++r) {
        const int jy = j0 + tg * 2 * NP + r;
        uint32_t key = kNoKey;
        if (col_ok && jy < R.ny) {
            int gpx = 0, gpy = 0;
            const int pix = pair_pixel(bxh[r], byh[r], bxl[r], byl[r], a.bin, gpx, gpy);
            if (pix >= 0) {
                ++nb;
                key = hist_key(pix, gpx, gpy, W, a.bin);
            } else if (pix == -1) {
                ++no;
            } else {
                ++nn;
            }
            if (a.beta_out) {
                float4 *bo = reinterpret_cast<float4 *>(a.beta_out);
                bo[(int64_t)jy * R.nx + ix] = make_float4(bxh[r], byh[r], bxl[r], byl[r]);
            }
        }
        hist_add_warp(key, W, a.counts);
    }
    __syncthreads();
    hist_flush(W, a.bin, a.counts);
    stats_add_block(nb, no, nn, ts.sred, a.stats);
}

}  // namespace mlens
