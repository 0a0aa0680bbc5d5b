// forecast_ns2d.cu -- batched SSP-RK3 forecast of the 2-D compressible
// Navier-Stokes equations (Eqs. Mass, Momentum, Energy) on periodic grids.
//
// State: 4 planes (rho, rho u, rho v, E) of n x n points, x fastest.  With
// u = (rho u)/rho, v = (rho v)/rho, p = (gamma-1)(E - rho |u|^2 / 2), T = p/rho:
//   dq/dt = -(F_{i+1} - F_{i-1}) / (2h) - (G_{j+1} - G_{j-1}) / (2h)
//           + (Fv_{i+1/2} - Fv_{i-1/2}) / h + (Gv_{j+1/2} - Gv_{j-1/2}) / h
// with nodal inviscid fluxes F = (rho u, rho u u + p, rho u v, (E + p) u),
// G = (rho v, rho v u, rho v v + p, (E + p) v) and face viscous/heat fluxes
// Fv = (0, t_xx, t_xy, t_xx u_f + t_xy v_f + kappa T_x) (normal derivatives
// compact across the face, tangential ones the average of the two central
// differences, face velocities the average of the two nodes), likewise Gv;
// t_xx = mu (4/3 u_x - 2/3 v_y), t_xy = mu (u_y + v_x), kappa = mu gamma /
// ((gamma - 1) Pr).  Every flux telescopes, so the four totals are conserved.
//
// GPU design: one launch per RK stage over every grid of the cycle (Ne members
// and the fine run).  A CTA owns a 32 x 8 tile: it loads the stage input of
// the tile and its one-point halo (periodic wrap) into shared memory, forms the
// primitives once per loaded point, and each thread evaluates the 9-point
// stencil of its point.  Stages: s1 = u0 + k(u0), s2 = u0 + ((s1 - u0) + k(s1))/4,
// u' = u0 + 2/3 ((s2 - u0) + k(s2)), k = dt L (Shu-Osher form rearranged);
// s1 and s2 live in two scratch buffers so a stage never overwrites a value
// another CTA still reads.
//
// FP32 states use a folded variant: a CTA of TX x H threads owns a TX x 2H
// tile and each thread the two points (x, y) and (x, y + H), held as one
// float2, so every shared-memory load is 64 bits wide and every arithmetic
// instruction is a packed FFMA2 / FADD2 / FMUL2 on both points; shared row r
// of the folded halo holds rows y0 + r - 1 and y0 + H + r - 1.  FP64 states
// use the scalar tile above.
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "forecast_ns2d.h"

namespace mgk {

constexpr int kNsTx = 32;
// tile rows of the per-handle kernel: 16 folded FP32 rows, 8 FP64 rows
template <typename T>
constexpr int ns_tile_rows() { return std::is_same<T, float>::value ? 16 : 8; }

template <typename T>
struct NsArgs {
    NsGroup<T> g[2];
    int tiles0;  // tiles of group 0
    T gm1, mu, kappa;
};

// The stencil body is written for a tile shape TX x TY (TX * TY = 256
// threads); the batched path picks the shape per grid size (autotuned).
template <typename T, int STAGE, int TX, int TY>
__device__ __forceinline__ void ns2d_stage_tile(const NsGroup<T> &G, int tile, T gm1, T mu, T kap) {
    constexpr int HX = TX + 2, HY = TY + 2, HALO = HX * HY;
    __shared__ T sq[4][HALO];   // conserved variables of the tile + halo
    __shared__ T spr[4][HALO];  // u, v, p, T
    const int tiles_per_prob = G.tx * G.ty;
    const int prob = tile / tiles_per_prob;
    const int tt = tile % tiles_per_prob;
    const int x0 = (tt % G.tx) * TX, y0 = (tt / G.tx) * TY;
    const int n = G.n;
    const size_t plane = (size_t)n * n;
    T *u0 = G.u0 + (size_t)prob * 4 * plane;
    const T *in = STAGE == 0 ? u0 : (STAGE == 1 ? G.s1 : G.s2) + (size_t)prob * 4 * plane;
    T *out = STAGE == 0 ? G.s1 + (size_t)prob * 4 * plane
                        : (STAGE == 1 ? G.s2 + (size_t)prob * 4 * plane : u0);

    // load the tile and its halo, form the primitives
    for (int e = threadIdx.x; e < HALO; e += blockDim.x) {
        const int ly = e / HX, lx = e % HX;
        int gy = y0 + ly - 1, gx = x0 + lx - 1;  // periodic wrap without integer division
        if (gy < 0) gy += n;
        if (gx < 0) gx += n;
        while (gy >= n) gy -= n;
        while (gx >= n) gx -= n;
        const size_t o = (size_t)gy * n + gx;
        const T rho = in[o], mx = in[plane + o], my = in[2 * plane + o], E = in[3 * plane + o];
        const T rinv = T(1) / rho;  // one division per point
        const T u = mx * rinv, v = my * rinv;
        const T p = gm1 * (E - T(0.5) * rho * (u * u + v * v));
        sq[0][e] = rho;
        sq[1][e] = mx;
        sq[2][e] = my;
        sq[3][e] = E;
        spr[0][e] = u;
        spr[1][e] = v;
        spr[2][e] = p;
        spr[3][e] = p * rinv;
    }
    __syncthreads();
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= n || y >= n) return;
    const int c = (ly + 1) * HX + (lx + 1);
    const int e_ = c + 1, w_ = c - 1, n_ = c + HX, s_ = c - HX;
    const T *U = spr[0], *V = spr[1], *P = spr[2], *TT = spr[3];
    const T ih = G.inv_h, i2h = G.inv_2h;
    const T c43 = T(4.0 / 3.0), c23 = T(2.0 / 3.0), half = T(0.5);
    // inviscid part: central differences of the nodal fluxes
    T r[4];
    {
        const T mxe = sq[1][e_], mxw = sq[1][w_], myn = sq[2][n_], mys = sq[2][s_];
        const T Fe1 = mxe * U[e_] + P[e_], Fw1 = mxw * U[w_] + P[w_];
        const T Fe2 = mxe * V[e_], Fw2 = mxw * V[w_];
        const T Fe3 = (sq[3][e_] + P[e_]) * U[e_], Fw3 = (sq[3][w_] + P[w_]) * U[w_];
        const T Gn1 = myn * U[n_], Gs1 = mys * U[s_];
        const T Gn2 = myn * V[n_] + P[n_], Gs2 = mys * V[s_] + P[s_];
        const T Gn3 = (sq[3][n_] + P[n_]) * V[n_], Gs3 = (sq[3][s_] + P[s_]) * V[s_];
        r[0] = -((mxe - mxw) + (myn - mys)) * i2h;
        r[1] = -((Fe1 - Fw1) + (Gn1 - Gs1)) * i2h;
        r[2] = -((Fe2 - Fw2) + (Gn2 - Gs2)) * i2h;
        r[3] = -((Fe3 - Fw3) + (Gn3 - Gs3)) * i2h;
    }
    // viscous and heat fluxes on the four faces of the node
    T fx[2][3], fy[2][3];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        {   // x-face between columns a = x-1+side and b = a+1
            const int a = side ? c : w_, b = side ? e_ : c;
            const T ux = (U[b] - U[a]) * ih, vx = (V[b] - V[a]) * ih;
            const T uy = half * ((U[a + HX] - U[a - HX]) + (U[b + HX] - U[b - HX])) * i2h;
            const T vy = half * ((V[a + HX] - V[a - HX]) + (V[b + HX] - V[b - HX])) * i2h;
            const T txx = mu * (c43 * ux - c23 * vy), txy = mu * (uy + vx);
            const T uf = half * (U[a] + U[b]), vf = half * (V[a] + V[b]);
            fx[side][0] = txx;
            fx[side][1] = txy;
            fx[side][2] = txx * uf + txy * vf + kap * (TT[b] - TT[a]) * ih;
        }
        {   // y-face between rows a = y-1+side and b = a+1
            const int a = side ? c : s_, b = side ? n_ : c;
            const T uy = (U[b] - U[a]) * ih, vy = (V[b] - V[a]) * ih;
            const T ux = half * ((U[a + 1] - U[a - 1]) + (U[b + 1] - U[b - 1])) * i2h;
            const T vx = half * ((V[a + 1] - V[a - 1]) + (V[b + 1] - V[b - 1])) * i2h;
            const T tyy = mu * (c43 * vy - c23 * ux), txy = mu * (uy + vx);
            const T uf = half * (U[a] + U[b]), vf = half * (V[a] + V[b]);
            fy[side][0] = txy;
            fy[side][1] = tyy;
            fy[side][2] = txy * uf + tyy * vf + kap * (TT[b] - TT[a]) * ih;
        }
    }
    T L[4];
    L[0] = r[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        L[k] = r[k] + ((fx[1][k - 1] - fx[0][k - 1]) + (fy[1][k - 1] - fy[0][k - 1])) * ih;

    const size_t o = (size_t)y * n + x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T kq = G.dt * L[k];
        const T s = sq[k][c];
        T res;
        if (STAGE == 0) {
            res = s + kq;
        } else {
            const T base = u0[k * plane + o];
            res = fma(STAGE == 1 ? T(0.25) : T(2.0 / 3.0), (s - base) + kq, base);
        }
        out[k * plane + o] = res;
    }
}

// ---------------------------------------------------------------------------
// FP32: folded pairs of points in float2, packed arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b with one rounding (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ int wrap_index(int g, int n) {
    if (g < 0) g += n;
    if (g >= n) {
        g -= n;
        if (g >= n) g %= n;  // only grids narrower than a tile
    }
    return g;
}

// 4-byte asynchronous global -> shared copy (cached in L1, where the halo
// re-reads of neighbouring tiles hit)
__device__ __forceinline__ void cp_async4(void *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// where the tiles of a launch come from: a device table of groups (batched
// path) or the two groups of one handle.  next() moves gi forward to the
// group holding `tile`; a CTA visits its tiles in increasing order.
struct TableTiles {
    const NsGroup<float> *groups;
    int ngroups;
    __device__ __forceinline__ void next(int tile, int &gi) const {
        while (gi + 1 < ngroups && groups[gi + 1].tile_begin <= tile) ++gi;
    }
    __device__ __forceinline__ NsGroup<float> group(int gi) const { return groups[gi]; }
};
struct PairTiles {
    NsGroup<float> g[2];  // g[1].tile_begin = tiles of g[0]
    __device__ __forceinline__ void next(int tile, int &gi) const { gi = tile < g[1].tile_begin ? 0 : 1; }
    // no runtime index into the parameter array
    __device__ __forceinline__ NsGroup<float> group(int gi) const { return gi ? g[1] : g[0]; }
};

// what every thread needs of one tile, prepared by thread 0 two tiles ahead
struct TileDesc {
    const float *in;  // stage input (4 planes of the grid)
    float *u0;        // state of the grid
    float *out;       // stage output
    int n, x0, y0, pad;
    float inv_h, inv_2h, dt, pad2;
};

template <int TX, int H, class Tiles>
__device__ __forceinline__ void make_desc(const Tiles &src, int tile, int &gi, int stage, TileDesc *d) {
    src.next(tile, gi);
    const NsGroup<float> G = src.group(gi);
    const int local = tile - G.tile_begin;
    const int tiles_per_prob = G.tx * G.ty;
    const int prob = local / tiles_per_prob;
    const int tt = local - prob * tiles_per_prob;
    const int ty = tt / G.tx;
    const int n = G.n;
    const size_t off = (size_t)prob * 4 * n * n;
    float *u0 = G.u0 + off;
    d->u0 = u0;
    d->in = stage == 0 ? u0 : (stage == 1 ? G.s1 : G.s2) + off;
    d->out = stage == 0 ? G.s1 + off : (stage == 1 ? G.s2 + off : u0);
    d->n = n;
    d->x0 = (tt - ty * G.tx) * TX;
    d->y0 = ty * (2 * H);
    d->inv_h = G.inv_h;
    d->inv_2h = G.inv_2h;
    d->dt = G.dt;
}

template <int TX, int H>
struct X2Smem {
    static constexpr int HX = TX + 2, HALO = HX * (H + 2), NT = TX * H;
    // raw halo: rows y0 - 1 .. y0 + 2H, columns x0 - 4 .. x0 + TX + 3 (16-byte
    // aligned), 4 planes, row-major
    static constexpr int RW = TX + 8, RR = 2 * H + 2, RAW = 4 * RR * RW;  // floats
    static constexpr int CHUNKS = 4 * RR * (RW / 4);                      // 16-byte copies per tile
    static constexpr int COPIES = (CHUNKS + NT - 1) / NT;                 // per thread
    // 2 raw buffers, 2 folded buffers of 8 arrays (rho, rho u, rho v, E, u, v, p, T), 4 descriptors
    static constexpr size_t bytes() {
        return sizeof(float) * 2 * RAW + sizeof(float2) * 2 * 8 * HALO + 4 * sizeof(TileDesc);
    }
};

// 16-byte asynchronous global -> shared copy (L2 only: each chunk is read once per tile)
__device__ __forceinline__ void cp_async16(void *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Issue the 16-byte copies of one tile's raw halo into one buffer.  Copy c of
// a thread is (plane, row, chunk); x0 - 4 and n are multiples of 4, so a
// chunk never straddles the periodic wrap.
template <int TX, int H>
__device__ __forceinline__ void x2_issue(const TileDesc &d, const int (&ck)[X2Smem<TX, H>::COPIES],
                                         const int (&cr)[X2Smem<TX, H>::COPIES],
                                         const int (&cx)[X2Smem<TX, H>::COPIES], float *raw) {
    using S = X2Smem<TX, H>;
    const int n = d.n, plane = n * n;  // 4 planes of one grid stay below 2^31 elements
#pragma unroll
    for (int q = 0; q < S::COPIES; ++q) {
        const int c = threadIdx.x + q * S::NT;
        if (c < S::CHUNKS) {
            const float *src = d.in + ck[q] * plane + wrap_index(d.y0 - 1 + cr[q], n) * n + wrap_index(d.x0 - 4 + cx[q], n);
            cp_async16(raw + (ck[q] * S::RR + cr[q]) * S::RW + cx[q], src);
        }
    }
}

__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Fold the raw halo and form the primitives: folded element e (row r, column
// lx) holds rows r and r + H of the raw block at column lx + 3.  Writes the 8
// folded arrays rho, rho u, rho v, E, u, v, p, T.
template <int TX, int H>
__device__ __forceinline__ void x2_fold(const float *raw, float2 *fold, float gm1) {
    using S = X2Smem<TX, H>;
    constexpr int HALO = S::HALO;
    for (int e = threadIdx.x; e < HALO; e += S::NT) {
        const int r = e / S::HX, lx = e - r * S::HX;
        const float *pa = raw + r * S::RW + lx + 3, *pb = pa + H * S::RW;
        const float2 rho = make_float2(pa[0], pb[0]);
        const float2 mx = make_float2(pa[S::RR * S::RW], pb[S::RR * S::RW]);
        const float2 my = make_float2(pa[2 * S::RR * S::RW], pb[2 * S::RR * S::RW]);
        const float2 E = make_float2(pa[3 * S::RR * S::RW], pb[3 * S::RR * S::RW]);
        const float2 rinv = make_float2(__fdividef(1.f, rho.x), __fdividef(1.f, rho.y));
        const float2 u = mul2(mx, rinv), v = mul2(my, rinv);
        const float2 ke = mul2(mul2(f2(0.5f), rho), fma2(u, u, mul2(v, v)));
        const float2 p = mul2(f2(gm1), sub2(E, ke));
        fold[e] = rho;
        fold[HALO + e] = mx;
        fold[2 * HALO + e] = my;
        fold[3 * HALO + e] = E;
        fold[4 * HALO + e] = u;
        fold[5 * HALO + e] = v;
        fold[6 * HALO + e] = p;
        fold[7 * HALO + e] = mul2(p, rinv);
    }
}

// dq/dt of the folded pair at shared index c (9-point stencil)
template <int HX, int HALO>
__device__ __forceinline__ void x2_rhs(const float2 *raw, const float2 *prim, int c, float inv_h, float inv_2h,
                                       float mu, float kap, float2 (&L)[4]) {
    const int e_ = c + 1, w_ = c - 1, n_ = c + HX, s_ = c - HX;
    const float2 *Q1 = raw + HALO, *Q2 = raw + 2 * HALO, *Q3 = raw + 3 * HALO;
    const float2 *U = prim, *V = prim + HALO, *P = prim + 2 * HALO, *TT = prim + 3 * HALO;
    const float2 ih = f2(inv_h), mi2h = f2(-inv_2h);
    float2 r[4];
    {   // inviscid part: central differences of the nodal fluxes
        const float2 mxe = Q1[e_], mxw = Q1[w_], myn = Q2[n_], mys = Q2[s_];
        const float2 Ue = U[e_], Uw = U[w_], Vn = V[n_], Vs = V[s_];
        const float2 Pe = P[e_], Pw = P[w_], Pn = P[n_], Ps = P[s_];
        const float2 Fe1 = fma2(mxe, Ue, Pe), Fw1 = fma2(mxw, Uw, Pw);
        const float2 Fe2 = mul2(mxe, V[e_]), Fw2 = mul2(mxw, V[w_]);
        const float2 Fe3 = mul2(add2(Q3[e_], Pe), Ue), Fw3 = mul2(add2(Q3[w_], Pw), Uw);
        const float2 Gn1 = mul2(myn, U[n_]), Gs1 = mul2(mys, U[s_]);
        const float2 Gn2 = fma2(myn, Vn, Pn), Gs2 = fma2(mys, Vs, Ps);
        const float2 Gn3 = mul2(add2(Q3[n_], Pn), Vn), Gs3 = mul2(add2(Q3[s_], Ps), Vs);
        r[0] = mul2(add2(sub2(mxe, mxw), sub2(myn, mys)), mi2h);
        r[1] = mul2(add2(sub2(Fe1, Fw1), sub2(Gn1, Gs1)), mi2h);
        r[2] = mul2(add2(sub2(Fe2, Fw2), sub2(Gn2, Gs2)), mi2h);
        r[3] = mul2(add2(sub2(Fe3, Fw3), sub2(Gn3, Gs3)), mi2h);
    }
    // viscous and heat fluxes on the four faces of the node.  The 1/h and
    // 1/(4h) of the derivatives sit in the stress coefficients, and the 1/2 of
    // the face velocities (and a factor 2 on the heat flux) in the final
    // 1/(2h) of the energy equation: the face fluxes of the discretisation,
    // with fewer multiplications.
    const float2 c43 = f2(4.f / 3.f), m16 = f2(-1.f / 6.f), q4 = f2(0.25f);
    const float2 k2 = f2(mu > 0.f ? 2.f * kap / mu : 0.f), mh2 = f2(mu * inv_h * inv_h), hmh2 = f2(0.5f * mu * inv_h * inv_h);
    float2 fx[2][3], fy[2][3];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        {   // x-face between columns a and b = a + 1
            const int a = side ? c : w_, b = side ? e_ : c;
            const float2 Ua = U[a], Ub = U[b], Va = V[a], Vb = V[b];
            const float2 dU = sub2(Ub, Ua), dV = sub2(Vb, Va);
            const float2 tU = add2(sub2(U[a + HX], U[a - HX]), sub2(U[b + HX], U[b - HX]));
            const float2 tV = add2(sub2(V[a + HX], V[a - HX]), sub2(V[b + HX], V[b - HX]));
            const float2 txx = fma2(c43, dU, mul2(m16, tV)), txy = fma2(q4, tU, dV);
            fx[side][0] = txx;
            fx[side][1] = txy;
            // 2 x (work + heat): txx (Ua + Ub) + txy (Va + Vb) + 2 kappa dT / h
            fx[side][2] = fma2(txx, add2(Ua, Ub), fma2(txy, add2(Va, Vb), mul2(k2, sub2(TT[b], TT[a]))));
        }
        {   // y-face between rows a and b = a + 1
            const int a = side ? c : s_, b = side ? n_ : c;
            const float2 Ua = U[a], Ub = U[b], Va = V[a], Vb = V[b];
            const float2 dU = sub2(Ub, Ua), dV = sub2(Vb, Va);
            const float2 tU = add2(sub2(U[a + 1], U[a - 1]), sub2(U[b + 1], U[b - 1]));
            const float2 tV = add2(sub2(V[a + 1], V[a - 1]), sub2(V[b + 1], V[b - 1]));
            const float2 tyy = fma2(c43, dV, mul2(m16, tU)), txy = fma2(q4, tV, dU);
            fy[side][0] = txy;
            fy[side][1] = tyy;
            fy[side][2] = fma2(txy, add2(Ua, Ub), fma2(tyy, add2(Va, Vb), mul2(k2, sub2(TT[b], TT[a]))));
        }
    }
    L[0] = r[0];
#pragma unroll
    for (int k = 1; k < 3; ++k)
        L[k] = fma2(add2(sub2(fx[1][k - 1], fx[0][k - 1]), sub2(fy[1][k - 1], fy[0][k - 1])), mh2, r[k]);
    L[3] = fma2(add2(sub2(fx[1][2], fx[0][2]), sub2(fy[1][2], fy[0][2])), hmh2, r[3]);
}

// Persistent stage kernel: each CTA walks tiles blockIdx.x, + gridDim.x, ...
// with one barrier per tile.  In iteration i it copies the raw halo of tile
// i + 2 (2 raw buffers), folds tile i + 1 and forms its primitives (2 folded
// buffers) and computes tile i; thread 0 describes tile i + 3 (4 descriptor
// slots).  Stages 1 and 2 load u0 at the thread's points at the start of the
// iteration and use it at the end.  At most 85 registers: three CTAs per SM.
template <int STAGE, int TX, int H, class Tiles>
__global__ void __launch_bounds__(256, 3) ns2d_stage_x2(Tiles src, int total_tiles, float gm1, float mu, float kap) {
    using S = X2Smem<TX, H>;
    constexpr int HX = S::HX, HALO = S::HALO, NT = S::NT;
    static_assert(NT == 256, "256 threads per CTA");
    extern __shared__ float4 x2_smem4[];
    float *raw_base = reinterpret_cast<float *>(x2_smem4);
    float2 *fold_base = reinterpret_cast<float2 *>(raw_base + 2 * S::RAW);
    TileDesc *desc = reinterpret_cast<TileDesc *>(fold_base + 2 * 8 * HALO);
    const int G = gridDim.x;
    // Stage launches follow one another with programmatic serialisation (see
    // x2_launch): the next stage may be scheduled from here on, and its CTAs
    // take the SMs as this launch's CTAs leave; each CTA prepares its first tile
    // descriptors (static tables only) before it waits for the previous launch
    // to complete and its writes to be visible.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    int tile = blockIdx.x;
    if (tile >= total_tiles) return;
    int gi = 0;  // thread 0: group of the last tile it described
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q)
            if (tile + q * G < total_tiles) make_desc<TX, H>(src, tile + q * G, gi, STAGE, &desc[q]);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int ck[S::COPIES], cr[S::COPIES], cx[S::COPIES];  // plane, raw row, first column of the thread's copies
#pragma unroll
    for (int q = 0; q < S::COPIES; ++q) {
        const int c = threadIdx.x + q * NT, row = c / (S::RW / 4), k = row / S::RR;
        ck[q] = k;
        cr[q] = row - k * S::RR;
        cx[q] = 4 * (c - row * (S::RW / 4));
    }
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    const int c = (ly + 1) * HX + (lx + 1);
    __syncthreads();
    x2_issue<TX, H>(desc[0], ck, cr, cx, raw_base);
    cp_async_commit();
    if (tile + G < total_tiles) x2_issue<TX, H>(desc[1], ck, cr, cx, raw_base + S::RAW);
    cp_async_commit();
    cp_async_wait1();  // tile 0's halo has landed
    __syncthreads();
    x2_fold<TX, H>(raw_base, fold_base, gm1);
    for (int it = 0; tile < total_tiles; ++it, tile += G) {
        cp_async_wait0();  // tile it + 1's halo has landed
        __syncthreads();   // publishes it and the folded tile it; iteration it - 1 is done everywhere
        const TileDesc &d = desc[it & 3];
        const int n = d.n, plane = n * n;
        const int x = d.x0 + lx, ya = d.y0 + ly, yb = ya + H;
        const bool ok = x < n && ya < n, has_b = ok && yb < n;
        float2 b[4];  // u0 at the thread's two points (stages 1, 2), consumed at the end of the iteration
        if (STAGE != 0) {
            const float *pa = d.u0 + (ok ? ya * n + x : 0);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                b[k] = make_float2(ok ? pa[k * plane] : 0.f, has_b ? pa[k * plane + H * n] : 0.f);
        }
        const bool has1 = tile + G < total_tiles, has2 = tile + 2 * G < total_tiles;
        if (threadIdx.x == 0 && tile + 3 * G < total_tiles) make_desc<TX, H>(src, tile + 3 * G, gi, STAGE, &desc[(it + 3) & 3]);
        // tile it + 2 goes to the raw buffer of tile it, folded in iteration it - 1
        if (has2) x2_issue<TX, H>(desc[(it + 2) & 3], ck, cr, cx, raw_base + (it & 1) * S::RAW);
        cp_async_commit();
        if (has1) x2_fold<TX, H>(raw_base + ((it + 1) & 1) * S::RAW, fold_base + ((it + 1) & 1) * 8 * HALO, gm1);
        const float2 *fq = fold_base + (it & 1) * 8 * HALO;

        if (ok) {
            float2 L[4];
            x2_rhs<HX, HALO>(fq, fq + 4 * HALO, c, d.inv_h, d.inv_2h, mu, kap, L);
            float *oa = d.out + ya * n + x, *ob = oa + H * n;
            const float2 dt = f2(d.dt);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 kq = mul2(dt, L[k]);
                const float2 sv = fq[k * HALO + c];
                float2 res;
                if (STAGE == 0)
                    res = add2(sv, kq);
                else
                    res = fma2(f2(STAGE == 1 ? 0.25f : 2.f / 3.f), add2(sub2(sv, b[k]), kq), b[k]);
                oa[k * plane] = res.x;
                if (has_b) ob[k * plane] = res.y;
            }
        }
    }
}

// CTAs per launch of a persistent stage kernel: resident CTAs per SM x SMs
template <int STAGE, int TX, int H, class Tiles>
static int x2_grid(int total_tiles) {
    static OncePerDevice once;
    static int ctas[kMaxDevices];  // resident CTAs per SM x SMs, per device
    once.run([](int dev) {
        const size_t smem = X2Smem<TX, H>::bytes();
        int per_sm = 0, sms = 0;
        cudaError_t e = cudaFuncSetAttribute(ns2d_stage_x2<STAGE, TX, H, Tiles>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ns2d_stage_x2<STAGE, TX, H, Tiles>, 256, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ctas[dev] = std::max(per_sm, 1) * std::max(sms, 1);
        return e;
    });
    const int dev = OncePerDevice::current();
    const int c = dev >= 0 && ctas[dev] > 0 ? ctas[dev] : kNumSMs;
    return std::min(total_tiles, c);
}

template <int STAGE, int TX, int H, class Tiles>
static void x2_launch(const Tiles &src, int total_tiles, float gm1, float mu, float kap, cudaStream_t s) {
    const int grid = x2_grid<STAGE, TX, H, Tiles>(total_tiles);
    // programmatic stream serialisation: the launch may start while the
    // previous kernel on the stream finishes; the kernel waits for it before
    // it touches the state (griddepcontrol.wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = X2Smem<TX, H>::bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, ns2d_stage_x2<STAGE, TX, H, Tiles>, src, total_tiles, gm1, mu, kap);
}

// per-handle FP64 launch: two groups (members, fine run) passed by value, 32 x 8 tiles
template <typename T, int STAGE>
__global__ void __launch_bounds__(256) ns2d_stage_kernel(NsArgs<T> A) {
    int tile = blockIdx.x;
    const int gi = tile < A.tiles0 ? 0 : 1;
    if (gi) tile -= A.tiles0;
    const NsGroup<T> G = gi ? A.g[1] : A.g[0];  // no runtime index into the parameter array
    ns2d_stage_tile<T, STAGE, 32, 8>(G, tile, A.gm1, A.mu, A.kappa);
}

const char *ns2d_check_size(int n_whole, int n_split) {
    for (int n : {n_whole, n_split}) {
        if (n < 8 || n > 4096 || n % 8 != 0) return "NS-2D grids need 8 <= n <= 4096 points per side with n % 8 == 0";
    }
    return nullptr;
}

size_t ns2d_scratch_elems(int n_whole, int n_whole_probs, int n_split, int n_split_probs) {
    return 2 * 4 * ((size_t)n_whole * n_whole * n_whole_probs + (size_t)n_split * n_split * n_split_probs);
}

template <typename T>
cudaError_t ns2d_forecast_scratch(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                                  int n_split_probs, double length, double dt, double mu,
                                  double gamma, double prandtl, int nsteps, T *scratch,
                                  cudaStream_t stream) {
    NsArgs<T> A = {};
    const int ns[2] = {n_whole, n_split}, np[2] = {n_whole_probs, n_split_probs};
    T *st[2] = {whole, split};
    T *sc = scratch;
    int tiles[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
        NsGroup<T> &G = A.g[g];
        G.n = ns[g];
        G.nprob = np[g];
        G.u0 = st[g];
        const size_t sz = (size_t)4 * ns[g] * ns[g] * np[g];
        G.s1 = sc;
        G.s2 = sc + sz;
        sc += 2 * sz;
        if (np[g] > 0) {
            G.tx = ceil_div(ns[g], kNsTx);
            G.ty = ceil_div(ns[g], ns_tile_rows<T>());
            const double h = length / ns[g];
            G.inv_h = (T)(1.0 / h);
            G.inv_2h = (T)(1.0 / (2.0 * h));
            G.dt = (T)dt;
            tiles[g] = G.tx * G.ty * np[g];
        }
    }
    A.tiles0 = tiles[0];
    A.gm1 = (T)(gamma - 1.0);
    A.mu = (T)mu;
    A.kappa = (T)(mu * gamma / ((gamma - 1.0) * prandtl));
    const int grid = tiles[0] + tiles[1];
    if (grid == 0 || nsteps == 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        // the halo is copied in 16-byte chunks
        if ((reinterpret_cast<uintptr_t>(whole) | reinterpret_cast<uintptr_t>(split) |
             reinterpret_cast<uintptr_t>(scratch)) & 15)
            return cudaErrorMisalignedAddress;
        PairTiles P{{A.g[0], A.g[1]}};
        P.g[0].tile_begin = 0;
        P.g[1].tile_begin = tiles[0];
        for (int s = 0; s < nsteps; ++s) {
            x2_launch<0, 32, 8>(P, grid, A.gm1, A.mu, A.kappa, stream);
            x2_launch<1, 32, 8>(P, grid, A.gm1, A.mu, A.kappa, stream);
            x2_launch<2, 32, 8>(P, grid, A.gm1, A.mu, A.kappa, stream);
            count_launches(3);
        }
    } else {
        for (int s = 0; s < nsteps; ++s) {
            ns2d_stage_kernel<T, 0><<<grid, 256, 0, stream>>>(A);
            ns2d_stage_kernel<T, 1><<<grid, 256, 0, stream>>>(A);
            ns2d_stage_kernel<T, 2><<<grid, 256, 0, stream>>>(A);
            count_launches(3);
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t ns2d_forecast(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                          int n_split_probs, double length, double dt, double mu, double gamma,
                          double prandtl, int nsteps, cudaStream_t stream) {
    // stream-ordered scratch for the stateless entry point
    const size_t elems = ns2d_scratch_elems(n_whole, n_whole_probs, n_split, n_split_probs);
    if (elems == 0 || nsteps == 0) return cudaSuccess;
    T *scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&scratch, elems * sizeof(T), stream);
    if (e != cudaSuccess) return e;
    e = ns2d_forecast_scratch<T>(whole, n_whole, n_whole_probs, split, n_split, n_split_probs, length, dt,
                                 mu, gamma, prandtl, nsteps, scratch, stream);
    cudaError_t e2 = cudaFreeAsync(scratch, stream);
    return e != cudaSuccess ? e : e2;
}

// batched FP32 shapes: threads TX x H, tiles TX x 2H points
int ns2d_tile_x(int shape) { return shape == 1 ? 16 : (shape == 2 ? 64 : 32); }
int ns2d_tile_y(int shape) { return 2 * (shape == 1 ? 16 : (shape == 2 ? 4 : 8)); }

template <int TX, int H>
static void launch_table(const NsGroup<float> *groups, int ngroups, int tiles, int nsteps, int first_stage,
                         int last_stage, float gm1, float mu, float kappa, cudaStream_t s) {
    const TableTiles src{groups, ngroups};
    for (int st = 0; st < nsteps; ++st) {
        for (int k = first_stage; k <= last_stage; ++k) {
            if (k == 0) x2_launch<0, TX, H>(src, tiles, gm1, mu, kappa, s);
            if (k == 1) x2_launch<1, TX, H>(src, tiles, gm1, mu, kappa, s);
            if (k == 2) x2_launch<2, TX, H>(src, tiles, gm1, mu, kappa, s);
        }
        count_launches(last_stage - first_stage + 1);
    }
}

static cudaError_t table_stages(const NsGroup<float> *d_groups, int ngroups, int tiles, int shape, int nsteps,
                                int first_stage, int last_stage, double gamma, double mu, double prandtl,
                                cudaStream_t s) {
    if (tiles == 0 || nsteps == 0) return cudaSuccess;
    const float gm1 = (float)(gamma - 1.0), m = (float)mu, kap = (float)(mu * gamma / ((gamma - 1.0) * prandtl));
    if (shape == 1)
        launch_table<16, 16>(d_groups, ngroups, tiles, nsteps, first_stage, last_stage, gm1, m, kap, s);
    else if (shape == 2)
        launch_table<64, 4>(d_groups, ngroups, tiles, nsteps, first_stage, last_stage, gm1, m, kap, s);
    else
        launch_table<32, 8>(d_groups, ngroups, tiles, nsteps, first_stage, last_stage, gm1, m, kap, s);
    return cudaGetLastError();
}

cudaError_t ns2d_forecast_table(const NsGroup<float> *d_groups, int ngroups, int tiles, int shape, int nsteps,
                                double gamma, double mu, double prandtl, cudaStream_t s) {
    return table_stages(d_groups, ngroups, tiles, shape, nsteps, 0, 2, gamma, mu, prandtl, s);
}

cudaError_t ns2d_probe_stages01(const NsGroup<float> *d_groups, int ngroups, int tiles, int shape, double gamma,
                                double mu, double prandtl, cudaStream_t s) {
    return table_stages(d_groups, ngroups, tiles, shape, 1, 0, 1, gamma, mu, prandtl, s);
}

#define MGK_NS_INST(T)                                                                            \
    template cudaError_t ns2d_forecast<T>(T *, int, int, T *, int, int, double, double, double,    \
                                          double, double, int, cudaStream_t);                     \
    template cudaError_t ns2d_forecast_scratch<T>(T *, int, int, T *, int, int, double, double,    \
                                                  double, double, double, int, T *, cudaStream_t); \

MGK_NS_INST(float)
MGK_NS_INST(double)
#undef MGK_NS_INST

}  // namespace mgk
