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
// GPU design, FP32 (the mixed path): one launch per time step over every grid
// of the cycle (Ne members and the fine run, or every grid of a batch), the
// three RK stages fused.  A persistent CTA walks tiles of TX x 2H points.  For
// each tile it copies the step-start state of the tile and a 3-point halo
// (periodic wrap) into shared memory, then evaluates stage 1 on the tile grown
// by 2 points, stage 2 on the tile grown by 1 and stage 3 on the tile, each
// stage reading the previous one from shared memory (the halo points are
// recomputed by the neighbouring tiles): per point and step the state is read
// once and written once.  Stages: s1 = u0 + k(u0), s2 = u0 + ((s1 - u0) +
// k(s1))/4, u' = u0 + 2/3 ((s2 - u0) + k(s2)), k = dt L (Shu-Osher form
// rearranged).  The step writes a second state buffer (a neighbouring tile may
// still read the old state's halo), so the steps alternate between the state
// and one scratch buffer; an odd step count ends with a copy back.
//
// Every thread works on pairs of points folded into float2: shared element
// (r, c) holds rows r and r + H of the tile's halo block, so every
// shared-memory access is 64 bits wide and every arithmetic instruction is a
// packed FFMA2 / FADD2 / FMUL2 on both points.
//
// FP64 states use one launch per stage: a CTA owns a 32 x 8 tile, loads the
// stage input of the tile and its one-point halo into shared memory, forms the
// primitives once per loaded point, and each thread evaluates the 9-point
// stencil of its point; s1 and s2 live in two scratch buffers.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "forecast_ns2d.h"

namespace mgk {

constexpr int kNsTx = 32;
// tile rows of the per-handle kernels: 32 FP32 rows (the fused step, 32 x 32
// points), 8 FP64 rows
template <typename T>
constexpr int ns_tile_rows() { return std::is_same<T, float>::value ? 32 : 8; }

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
// FP32: folded pairs of points in float2, packed arithmetic, fused RK stages
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b with one rounding (packed subtraction; no constant operand)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
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

// 16-byte asynchronous global -> shared copy (L2 only: each chunk is read once per tile)
__device__ __forceinline__ void cp_async16(void *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// The FP32 step on 2-D tiles (the per-handle path: the members and the fine
// run in one persistent launch).  A CTA walks tiles of TX x 2H points; for each
// it copies the step-start state of the tile and a 3-point halo into shared
// memory, evaluates stage 1 on the tile grown by 2 points, stage 2 on the
// tile grown by 1 and stage 3 on the tile, each stage reading the previous
// one from shared memory.  Shared element (r, c) holds rows r and r + H of the
// halo block (one float2).
// ---------------------------------------------------------------------------
// where the tiles of a launch come from: a device table of groups (batched
// path) or the two groups of one handle.  next() moves gi forward to the
// group holding `tile`; a CTA visits its tiles in increasing order.
struct PairTiles {
    NsGroup<float> g[2];  // g[1].tile_begin = tiles of g[0]
    __device__ __forceinline__ void next(int tile, int &gi) const { gi = tile < g[1].tile_begin ? 0 : 1; }
    // no runtime index into the parameter array
    __device__ __forceinline__ NsGroup<float> group(int gi) const { return gi ? g[1] : g[0]; }
};

// what every thread needs of one tile, prepared by thread 0 two tiles ahead
struct TileDesc {
    const float *in;  // step-start state (4 planes of the grid)
    float *out;       // state after the step
    int n, x0, y0, pad;
    float inv_h, inv_2h, dt, pad2;
};

// Steps alternate between the grid's state (u0) and its scratch buffer (s1):
// parity 0 reads u0 and writes s1, parity 1 the reverse.
template <int TX, int H, class Tiles>
__device__ __forceinline__ void make_desc(const Tiles &src, int tile, int &gi, int parity, TileDesc *d) {
    src.next(tile, gi);
    const NsGroup<float> G = src.group(gi);
    const int local = tile - G.tile_begin;
    const int tiles_per_prob = G.tx * G.ty;
    const int prob = local / tiles_per_prob;
    const int tt = local - prob * tiles_per_prob;
    const int ty = tt / G.tx;
    const int n = G.n;
    const size_t off = (size_t)prob * 4 * n * n;
    float *u0 = G.u0 + off, *other = G.s1 + off;
    d->in = parity ? other : u0;
    d->out = parity ? u0 : other;
    d->n = n;
    d->x0 = (tt - ty * G.tx) * TX;
    d->y0 = ty * (2 * H);
    d->inv_h = G.inv_h;
    d->inv_2h = G.inv_2h;
    d->dt = G.dt;
}

// dq/dt of the folded pair at shared index c (9-point stencil); `cons` holds
// the conserved planes (rho, rho u, rho v, E), `prim` u, v, p, T, each HALO
// elements long
template <int HX, int HALO>
__device__ __forceinline__ void x2_rhs(const float2 *cons, const float2 *prim, int c, float inv_h, float inv_2h,
                                       float mu, float kap, float2 (&L)[4]) {
    const int e_ = c + 1, w_ = c - 1, n_ = c + HX, s_ = c - HX;
    const float2 *Q1 = cons + HALO, *Q2 = cons + 2 * HALO, *Q3 = cons + 3 * HALO;
    const float2 *U = prim, *V = prim + HALO, *P = prim + 2 * HALO, *TT = prim + 3 * HALO;
    const float2 mi2h = f2(-inv_2h);
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

// primitives u, v, p, T of a folded pair of conserved values (one approximate
// reciprocal of rho per point)
template <int HALO>
__device__ __forceinline__ void put_prims(float2 *prim, int f, float2 rho, float2 mx, float2 my, float2 E, float gm1) {
    const float2 rinv = make_float2(__fdividef(1.f, rho.x), __fdividef(1.f, rho.y));
    const float2 u = mul2(mx, rinv), v = mul2(my, rinv);
    const float2 ke = mul2(mul2(f2(0.5f), rho), fma2(u, u, mul2(v, v)));
    const float2 p = mul2(f2(gm1), sub2(E, ke));
    prim[f] = u;
    prim[HALO + f] = v;
    prim[2 * HALO + f] = p;
    prim[3 * HALO + f] = mul2(p, rinv);
}

// Shared memory of the fused step for tiles of TX x 2H points (TX x H folded
// pairs) with a 3-point halo.
template <int TX, int H>
struct StepSmem {
    static constexpr int NT = 256;                 // threads per CTA
    static constexpr int FX = TX + 6, FR = H + 6;  // folded block: columns x0-3 .., rows r and r + H of rows y0-3 ..
    static constexpr int NF = FX * FR;             // folded elements per array
    // raw block of the step-start state: rows y0 - 3 .. y0 + 2H + 2, columns
    // x0 - 4 .. x0 + TX + 3 (16-byte aligned), 4 planes, row-major
    static constexpr int RW = TX + 8, RR = 2 * H + 6, RAW = 4 * RR * RW;  // floats
    static constexpr int CHUNKS = 4 * RR * (RW / 4);                      // 16-byte copies per tile
    static constexpr int COPIES = (CHUNKS + NT - 1) / NT;                 // per thread
    // u0 (4 arrays), the current stage (4), its primitives (4), raw block, 4 descriptors
    static constexpr size_t bytes() { return sizeof(float2) * 12 * NF + sizeof(float) * RAW + 4 * sizeof(TileDesc); }
    static_assert((TX * H) % NT == 0, "the last stage gives every thread the same number of pairs");
};

// Issue the 16-byte copies of one tile's raw block.  Copy c of a thread is
// (plane, row, chunk); x0 - 4 and n are multiples of 4, so a chunk never
// straddles the periodic wrap.
template <int TX, int H>
__device__ __forceinline__ void step_issue(const TileDesc &d, float *raw) {
    using S = StepSmem<TX, H>;
    const int n = d.n, plane = n * n;  // 4 planes of one grid stay below 2^31 elements
#pragma unroll
    for (int q = 0; q < S::COPIES; ++q) {
        const int c = threadIdx.x + q * S::NT;
        if (c < S::CHUNKS) {
            // plane k, raw row r, first column x of the chunk (divisions by constants)
            const int row = c / (S::RW / 4), k = row / S::RR, r = row - k * S::RR, x = 4 * (c - row * (S::RW / 4));
            const float *src = d.in + k * plane + wrap_index(d.y0 - 3 + r, n) * n + wrap_index(d.x0 - 4 + x, n);
            cp_async16(raw + row * S::RW + x, src);
        }
    }
}

// Fold the raw block (folded element (r, c) holds raw rows r and r + H at raw
// column c + 1) into u0 and form its primitives.
template <int TX, int H>
__device__ __forceinline__ void step_fold(const float *raw, float2 *Q0, float2 *PR, float gm1) {
    using S = StepSmem<TX, H>;
    constexpr int NF = S::NF, PL = S::RR * S::RW;
    for (int e = threadIdx.x; e < NF; e += S::NT) {
        const int r = e / S::FX, c = e - r * S::FX;
        const float *pa = raw + r * S::RW + c + 1, *pb = pa + H * S::RW;
        const float2 rho = make_float2(pa[0], pb[0]);
        const float2 mx = make_float2(pa[PL], pb[PL]);
        const float2 my = make_float2(pa[2 * PL], pb[2 * PL]);
        const float2 E = make_float2(pa[3 * PL], pb[3 * PL]);
        Q0[e] = rho;
        Q0[NF + e] = mx;
        Q0[2 * NF + e] = my;
        Q0[3 * NF + e] = E;
        put_prims<NF>(PR, e, rho, mx, my, E, gm1);
    }
}

// Stage K (1 or 2) on the folded block shrunk by K on every side: reads the
// previous stage (u0 for K = 1) and its primitives, and after a barrier
// replaces them with this stage's values (the results wait in registers).
template <int TX, int H, int K>
__device__ __forceinline__ void step_stage(const float2 *Q0, float2 *QS, float2 *PR, const TileDesc &d, float gm1,
                                           float mu, float kap) {
    using S = StepSmem<TX, H>;
    constexpr int W = S::FX - 2 * K, R = S::FR - 2 * K, N = W * R, E = (N + S::NT - 1) / S::NT, NF = S::NF;
    const float2 *cons = K == 1 ? Q0 : QS;
    const float2 dt = f2(d.dt);
    float2 res[E][4];
    int fo[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int e = threadIdx.x + q * S::NT;
        fo[q] = -1;
        if (e < N) {
            const int r = e / W, c = e - r * W;
            const int f = (r + K) * S::FX + c + K;
            fo[q] = f;
            float2 L[4];
            x2_rhs<S::FX, NF>(cons, PR, f, d.inv_h, d.inv_2h, mu, kap, L);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 kq = mul2(dt, L[k]);
                const float2 base = Q0[k * NF + f];
                res[q][k] = K == 1 ? add2(base, kq) : fma2(f2(0.25f), add2(sub2(QS[k * NF + f], base), kq), base);
            }
        }
    }
    __syncthreads();  // every read of the previous stage is done
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int f = fo[q];
        if (f >= 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) QS[k * NF + f] = res[q][k];
            put_prims<NF>(PR, f, res[q][0], res[q][1], res[q][2], res[q][3], gm1);
        }
    }
    __syncthreads();  // this stage is complete
}

// Stage 3 on the tile itself, straight to the output state.
template <int TX, int H>
__device__ __forceinline__ void step_last(const float2 *Q0, const float2 *QS, const float2 *PR, const TileDesc &d,
                                          float mu, float kap) {
    using S = StepSmem<TX, H>;
    constexpr int E = TX * H / S::NT, NF = S::NF;
    const float2 dt = f2(d.dt);
    const int n = d.n, plane = n * n;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int e = threadIdx.x + q * S::NT;
        const int r = e / TX, c = e - r * TX;
        const int f = (r + 3) * S::FX + c + 3;
        const int x = d.x0 + c, ya = d.y0 + r, yb = ya + H;
        if (x >= n || ya >= n) continue;
        float2 L[4];
        x2_rhs<S::FX, NF>(QS, PR, f, d.inv_h, d.inv_2h, mu, kap, L);
        float *oa = d.out + ya * n + x, *ob = oa + H * n;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 kq = mul2(dt, L[k]);
            const float2 base = Q0[k * NF + f];
            const float2 res = fma2(f2(2.f / 3.f), add2(sub2(QS[k * NF + f], base), kq), base);
            oa[k * plane] = res.x;
            if (yb < n) ob[k * plane] = res.y;
        }
    }
}

// One SSP-RK3 step of every tile of a launch.  Persistent: each CTA walks
// tiles blockIdx.x, + gridDim.x, ...; the raw block of the next tile is
// copied while the three stages of the current one run; thread 0 describes
// tiles two ahead (4 descriptor slots).
template <int TX, int H, int MINB, class Tiles>
__global__ void __launch_bounds__(256, MINB)
    ns2d_rk3_step(Tiles src, int total_tiles, int parity, float gm1, float mu, float kap) {
    using S = StepSmem<TX, H>;
    constexpr int NF = S::NF;
    extern __shared__ float4 step_smem4[];
    float2 *Q0 = reinterpret_cast<float2 *>(step_smem4);
    float2 *QS = Q0 + 4 * NF;
    float2 *PR = QS + 4 * NF;
    float *raw = reinterpret_cast<float *>(PR + 4 * NF);
    TileDesc *desc = reinterpret_cast<TileDesc *>(raw + S::RAW);
    const int G = gridDim.x;
    // Steps follow one another with programmatic serialisation (see
    // step_launch): the next step may be scheduled from here on, and its CTAs
    // take the SMs as this launch's CTAs leave; each CTA describes its first
    // tiles (static tables only) before it waits for the previous launch to
    // complete and its writes to be visible.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    int tile = blockIdx.x;
    if (tile >= total_tiles) return;
    int gi = 0;  // thread 0: group of the last tile it described
    if (threadIdx.x == 0)
        for (int q = 0; q < 2; ++q)
            if (tile + q * G < total_tiles) make_desc<TX, H>(src, tile + q * G, gi, parity, &desc[q]);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();
    step_issue<TX, H>(desc[0], raw);
    cp_async_commit();
    for (int it = 0; tile < total_tiles; ++it, tile += G) {
        cp_async_wait0();  // this tile's raw block has landed
        __syncthreads();   // ... for every thread; the previous tile is done everywhere
        step_fold<TX, H>(raw, Q0, PR, gm1);
        __syncthreads();   // the raw block is free, u0 and its primitives are ready
        if (tile + G < total_tiles) step_issue<TX, H>(desc[(it + 1) & 3], raw);
        cp_async_commit();
        if (threadIdx.x == 0 && tile + 2 * G < total_tiles)
            make_desc<TX, H>(src, tile + 2 * G, gi, parity, &desc[(it + 2) & 3]);
        const TileDesc &d = desc[it & 3];
        step_stage<TX, H, 1>(Q0, QS, PR, d, gm1, mu, kap);
        step_stage<TX, H, 2>(Q0, QS, PR, d, gm1, mu, kap);
        step_last<TX, H>(Q0, QS, PR, d, mu, kap);
    }
}

// ---------------------------------------------------------------------------
// The FP32 step as a column march.  A CTA owns a band of columns of one grid
// and a segment of its rows; thread t owns the column pair (c0 + t, c0 + t +
// T) as one float2 (T = blockDim.x).  With one band the pair spans the whole
// periodic width (c0 = 0, 2T = n); with several bands (n > 512) each band
// carries a 3-column halo on both sides, recomputed by its neighbours.  The
// CTA marches down the rows of its segment: in step j it loads row j of the
// step-start state (3 rows above the segment first), evaluates stage 1 one row
// behind, stage 2 three rows behind and stage 3 five rows behind, and stores
// the new state's row.  Each stage keeps the three rows of its input around
// the row it evaluates in registers (its own columns); only the east and west
// neighbours come from shared memory, through ring buffers of the last rows
// each stage published (one barrier per step).  The face between two rows is
// evaluated once and carried to the next row.
// ---------------------------------------------------------------------------
// one row of a stage input at the thread's column pair
struct Rec {
    float2 rho, mx, my, E, U, V, P, T;
};

// primitives u, v, p, T of a pair of conserved values (one approximate
// reciprocal of rho per point)
__device__ __forceinline__ Rec make_rec(float2 rho, float2 mx, float2 my, float2 E, float gm1) {
    Rec r;
    r.rho = rho;
    r.mx = mx;
    r.my = my;
    r.E = E;
    const float2 rinv = make_float2(__fdividef(1.f, rho.x), __fdividef(1.f, rho.y));
    r.U = mul2(mx, rinv);
    r.V = mul2(my, rinv);
    const float2 ke = mul2(mul2(f2(0.5f), rho), fma2(r.U, r.U, mul2(r.V, r.V)));
    r.P = mul2(f2(gm1), sub2(E, ke));
    r.T = mul2(r.P, rinv);
    return r;
}

// Viscous and heat fluxes of one face, in units of mu/h (pure-number stress
// coefficients; the 1/2 of the face velocities and a factor 2 on the heat
// flux are in the final 1/(2h) of the energy equation).  tU, tV: sums of the
// two central tangential differences of u and v across the face.
struct Face {
    float2 f0, f1, f2;
};
// x-face between columns a and b = a + 1: (t_xx, t_xy, 2 x (work + heat))
__device__ __forceinline__ Face face_x(float2 Ua, float2 Ub, float2 Va, float2 Vb, float2 tU, float2 tV, float2 Ta,
                                       float2 Tb, float2 k2) {
    const float2 dU = sub2(Ub, Ua), dV = sub2(Vb, Va);
    const float2 txx = fma2(f2(4.f / 3.f), dU, mul2(f2(-1.f / 6.f), tV)), txy = fma2(f2(0.25f), tU, dV);
    Face F;
    F.f0 = txx;
    F.f1 = txy;
    F.f2 = fma2(txx, add2(Ua, Ub), fma2(txy, add2(Va, Vb), mul2(k2, sub2(Tb, Ta))));
    return F;
}
// y-face between rows a and b = a + 1: (t_xy, t_yy, 2 x (work + heat))
__device__ __forceinline__ Face face_y(float2 Ua, float2 Ub, float2 Va, float2 Vb, float2 tU, float2 tV, float2 Ta,
                                       float2 Tb, float2 k2) {
    const float2 dU = sub2(Ub, Ua), dV = sub2(Vb, Va);
    const float2 tyy = fma2(f2(4.f / 3.f), dV, mul2(f2(-1.f / 6.f), tU)), txy = fma2(f2(0.25f), tV, dU);
    Face F;
    F.f0 = txy;
    F.f1 = tyy;
    F.f2 = fma2(txy, add2(Ua, Ub), fma2(tyy, add2(Va, Vb), mul2(k2, sub2(Tb, Ta))));
    return F;
}

// Shared ring buffers of the march, float2 per thread (T threads; each ring
// row holds T + 2 pairs: slot t + 1 is thread t's pair, slot 0 the last
// thread's pair and slot T + 1 the first thread's pair, both with their halves
// swapped, so that the east and west neighbours across the fold are plain
// loads):
//   rows [4k + s]:           u of stage input k (k = 0 u0, 1 s1, 2 s2), ring slot s of 4
//   rows [12 + 4k + s]:      v
//   rows [24 + 12k + 3f + s]: rho u, E, p, T (f = 0..3) of stage input k, ring slot s of 3
//   rows [60 + 4s + f]:      rho, rho u, rho v, E of u0, ring slot s of 8 (own column only)
constexpr int kMarchRows = 92;
// shared bytes of a march CTA of T threads
__host__ __device__ __forceinline__ size_t march_smem_bytes(int threads) {
    return sizeof(float2) * kMarchRows * (size_t)(threads + 2);
}
constexpr int kMarchMaxThreads = 256;
constexpr int kMarchBandMax = 2 * kMarchMaxThreads - 6;  // output columns of a band (even)
constexpr int kMarchNarrowBand = 122;  // output columns of a narrow band: 64 threads per CTA

// Thread t's slot in a ring row (row pitch T + 2), and the slot that holds its
// pair swapped for the thread at the other end of the fold (-1: none).
struct Slot {
    int own, mirror;
};

__device__ __forceinline__ void put_pair(float2 *row, const Slot &sl, float2 v) {
    row[sl.own] = v;
    if (sl.mirror >= 0) row[sl.mirror] = make_float2(v.y, v.x);
}

__device__ __forceinline__ void march_publish(float2 *X, int P, const Slot &sl, int k, int j, const Rec &r) {
    put_pair(X + (4 * k + (j & 3)) * P, sl, r.U);
    put_pair(X + (12 + 4 * k + (j & 3)) * P, sl, r.V);
    float2 *F = X + (24 + 12 * k + j % 3) * P;
    put_pair(F, sl, r.mx);
    put_pair(F + 3 * P, sl, r.E);
    put_pair(F + 6 * P, sl, r.P);
    put_pair(F + 9 * P, sl, r.T);
}

// east / west neighbour of the thread's pair in a ring row: the pair of thread
// t + 1 (t - 1), across the fold the mirrored pair of the other end
struct Nbr {
    int te, tw;  // slots t + 2 and t
    __device__ __forceinline__ float2 e(const float2 *row) const { return row[te]; }
    __device__ __forceinline__ float2 w(const float2 *row) const { return row[tw]; }
};

// Stage input k, evaluated in step j at the centre row c of the window
// (T: ring row pitch)
// (m1, c, p1 published in steps j - 2, j - 1, j).  yf: in, the face between
// m1 and c (carried from the previous step); out, the face between c and p1.
// FULL = false computes only that face (the step before a stage's first row).
template <bool FULL>
__device__ __forceinline__ void march_rhs(const float2 *X, int T, const Nbr &nb, int k, int j, const Rec &m1,
                                          const Rec &c, const Rec &p1, float inv_h, float inv_2h, float mu,
                                          float kap, Face &yf, float2 (&L)[4]) {
    const float2 *XU = X + 4 * k * T, *XV = X + (12 + 4 * k) * T;
    const int sm = ((j - 2) & 3) * T, sc = ((j - 1) & 3) * T, sp = (j & 3) * T;
    const float2 k2 = f2(mu > 0.f ? 2.f * kap / mu : 0.f);
    const float2 Uec = nb.e(XU + sc), Uwc = nb.w(XU + sc), Vec = nb.e(XV + sc), Vwc = nb.w(XV + sc);
    const float2 Uep = nb.e(XU + sp), Uwp = nb.w(XU + sp), Vep = nb.e(XV + sp), Vwp = nb.w(XV + sp);
    // face between c and p1
    const Face top = face_y(c.U, p1.U, c.V, p1.V, add2(sub2(Uec, Uwc), sub2(Uep, Uwp)),
                            add2(sub2(Vec, Vwc), sub2(Vep, Vwp)), c.T, p1.T, k2);
    if (FULL) {
        const float2 Uem = nb.e(XU + sm), Uwm = nb.w(XU + sm), Vem = nb.e(XV + sm), Vwm = nb.w(XV + sm);
        const float2 *XF = X + (24 + 12 * k + (j - 1) % 3) * T;
        const float2 mxe = nb.e(XF), mxw = nb.w(XF), Ee = nb.e(XF + 3 * T), Ew = nb.w(XF + 3 * T);
        const float2 Pe = nb.e(XF + 6 * T), Pw = nb.w(XF + 6 * T), Te = nb.e(XF + 9 * T), Tw = nb.w(XF + 9 * T);
        // inviscid part: central differences of the nodal fluxes
        const float2 mi2h = f2(-inv_2h);
        const float2 myn = p1.my, mys = m1.my;
        const float2 Fe1 = fma2(mxe, Uec, Pe), Fw1 = fma2(mxw, Uwc, Pw);
        const float2 Fe2 = mul2(mxe, Vec), Fw2 = mul2(mxw, Vwc);
        const float2 Fe3 = mul2(add2(Ee, Pe), Uec), Fw3 = mul2(add2(Ew, Pw), Uwc);
        const float2 Gn1 = mul2(myn, p1.U), Gs1 = mul2(mys, m1.U);
        const float2 Gn2 = fma2(myn, p1.V, p1.P), Gs2 = fma2(mys, m1.V, m1.P);
        const float2 Gn3 = mul2(add2(p1.E, p1.P), p1.V), Gs3 = mul2(add2(m1.E, m1.P), m1.V);
        const float2 r0 = mul2(add2(sub2(mxe, mxw), sub2(myn, mys)), mi2h);
        const float2 r1 = mul2(add2(sub2(Fe1, Fw1), sub2(Gn1, Gs1)), mi2h);
        const float2 r2 = mul2(add2(sub2(Fe2, Fw2), sub2(Gn2, Gs2)), mi2h);
        const float2 r3 = mul2(add2(sub2(Fe3, Fw3), sub2(Gn3, Gs3)), mi2h);
        // x-faces of the centre row
        const Face fw = face_x(Uwc, c.U, Vwc, c.V, add2(sub2(Uwp, Uwm), sub2(p1.U, m1.U)),
                               add2(sub2(Vwp, Vwm), sub2(p1.V, m1.V)), Tw, c.T, k2);
        const Face fe = face_x(c.U, Uec, c.V, Vec, add2(sub2(p1.U, m1.U), sub2(Uep, Uem)),
                               add2(sub2(p1.V, m1.V), sub2(Vep, Vem)), c.T, Te, k2);
        const float2 mh2 = f2(mu * inv_h * inv_h), hmh2 = f2(0.5f * mu * inv_h * inv_h);
        L[0] = r0;
        L[1] = fma2(add2(sub2(fe.f0, fw.f0), sub2(top.f0, yf.f0)), mh2, r1);
        L[2] = fma2(add2(sub2(fe.f1, fw.f1), sub2(top.f1, yf.f1)), mh2, r2);
        L[3] = fma2(add2(sub2(fe.f2, fw.f2), sub2(top.f2, yf.f2)), hmh2, r3);
    }
    yf = top;
}

// one unit of a march launch: a band and a row segment of one grid
struct MarchUnit {
    const float *in;  // step-start state of the grid (4 planes)
    float *out;       // state after the step
    int n, c0, y0, rows;  // points per side, first column (may be negative), first row, rows of the segment
    int ilo, ihi;         // output columns: pair index i (t or t + T) in [ilo, ihi)
    float inv_h, inv_2h, dt;
};

// bands and row segments of one n x n grid (host and device agree)
// bands of at most kMarchBandMax columns (the whole width up to 512), or
// with `narrow` of at most kMarchNarrowBand (the whole width up to 128)
__host__ __device__ __forceinline__ int march_bands(int n, bool narrow = false) {
    if (narrow) return n <= 128 ? 1 : (n + kMarchNarrowBand - 1) / kMarchNarrowBand;
    return n <= 2 * kMarchMaxThreads ? 1 : (n + kMarchBandMax - 1) / kMarchBandMax;
}
__host__ __device__ __forceinline__ int march_band_width(int n, int bands) {
    if (bands == 1) return n;
    const int w = (n + bands - 1) / bands;
    return w + (w & 1);
}
__host__ __device__ __forceinline__ int march_threads(int n, bool narrow = false) {
    const int b = march_bands(n, narrow);
    return b == 1 ? n / 2 : (march_band_width(n, b) + 6) / 2;
}

__device__ __forceinline__ MarchUnit march_unit(const NsGroup<float> &G, int local, int parity) {
    const int per_grid = G.tx * G.ty;
    const int prob = local / per_grid;
    const int rem = local - prob * per_grid;
    const int band = rem / G.ty, seg = rem - band * G.ty;
    const int n = G.n;
    const size_t off = (size_t)prob * 4 * n * n;
    float *u0 = G.u0 + off, *other = G.s1 + off;
    MarchUnit u;
    u.in = parity ? other : u0;
    u.out = parity ? u0 : other;
    u.n = n;
    const int S = (n + G.ty - 1) / G.ty;
    u.y0 = seg * S;
    u.rows = min(S, n - u.y0);
    if (G.tx == 1) {
        u.c0 = 0;
        u.ilo = 0;
        u.ihi = n;
    } else {
        const int bw = march_band_width(n, G.tx), bx0 = band * bw;
        u.c0 = bx0 - 3;
        u.ilo = 3;
        u.ihi = 3 + min(bw, n - bx0);
    }
    u.inv_h = G.inv_h;
    u.inv_2h = G.inv_2h;
    u.dt = G.dt;
    return u;
}

// where the units of a launch come from: a device table of groups of one grid
// size (batched path) or one group passed by value
struct TableUnits {
    const NsGroup<float> *groups;
    int ngroups;
    __device__ __forceinline__ MarchUnit unit(int u, int parity) const {
        int gi = 0;
        while (gi + 1 < ngroups && groups[gi + 1].tile_begin <= u) ++gi;
        const NsGroup<float> G = groups[gi];
        return march_unit(G, u - G.tile_begin, parity);
    }
    __device__ __forceinline__ NsGroup<float> group(int gi) const { return groups[gi]; }
};
struct OneUnits {
    NsGroup<float> g;
    __device__ __forceinline__ MarchUnit unit(int u, int parity) const { return march_unit(g, u, parity); }
    __device__ __forceinline__ NsGroup<float> group(int) const { return g; }
};

// One SSP-RK3 step of one unit per CTA (blockDim.x = march_threads(n) of the
// launch's grid size).  Step j of the march: rows of u0 arrive in steps
// 0 .. rows + 5 (rows y0 - 3 .. y0 + rows + 2); stage 1 evaluates row
// y0 - 4 + j in steps 2 .. rows + 5, stage 2 row y0 - 6 + j in steps
// 5 .. rows + 6, stage 3 row y0 - 8 + j in steps 8 .. rows + 7; a stage's
// output row is published one step after it is computed.
template <class Units>
__global__ void __launch_bounds__(kMarchMaxThreads, 1)
    ns2d_rk3_march(Units src, int parity, float gm1, float mu, float kap) {
    extern __shared__ float4 march_smem4[];
    float2 *X = reinterpret_cast<float2 *>(march_smem4);
    const int T = blockDim.x, t = threadIdx.x, P = T + 2;  // threads, ring row pitch
    // Steps follow one another with programmatic serialisation (see
    // march_launch): the next step may be scheduled from here on; each CTA
    // decodes its unit (static tables only) before it waits for the previous
    // launch to complete and its writes to be visible.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const MarchUnit u = src.unit(blockIdx.x, parity);
    Nbr nb;
    nb.te = t + 2;
    nb.tw = t;
    Slot sl;
    sl.own = t + 1;
    sl.mirror = t == 0 ? T + 1 : (t == T - 1 ? 0 : -1);
    if (T == 1) sl.mirror = -1;  // never: T = n/2 >= 4
    const int n = u.n, plane = n * n;  // 4 planes of one grid stay below 2^31 elements
    const int xa = wrap_index(u.c0 + t, n), xb = wrap_index(u.c0 + t + T, n);
    const bool wa = t >= u.ilo && t < u.ihi, wb = t + T >= u.ilo && t + T < u.ihi;
    const int R = u.rows;
    asm volatile("griddepcontrol.wait;" ::: "memory");

    float ld[8];  // the next u0 row at the two columns: rho, rho u, rho v, E
    auto load_row = [&](int j) {
        const float *p = u.in + wrap_index(u.y0 - 3 + j, n) * n;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ld[2 * q] = __ldg(p + q * plane + xa);
            ld[2 * q + 1] = __ldg(p + q * plane + xb);
        }
    };
    load_row(0);
    const float2 dt = f2(u.dt);
    Rec a_m1{}, a_c{}, a_p1{};  // u0 rows around stage 1's row
    Rec b_m1{}, b_c{}, b_p1{};  // s1 rows around stage 2's row
    Rec c_m1{}, c_c{}, c_p1{};  // s2 rows around stage 3's row
    Face yf1{}, yf2{}, yf3{};   // carried faces
    float2 L[4];
    const int steps = R + 8;
    for (int j = 0; j < steps; ++j) {
        // publish the rows that arrive in this step
        if (j <= R + 5) {
            const Rec r = make_rec(make_float2(ld[0], ld[1]), make_float2(ld[2], ld[3]), make_float2(ld[4], ld[5]),
                                   make_float2(ld[6], ld[7]), gm1);
            a_m1 = a_c;
            a_c = a_p1;
            a_p1 = r;
            march_publish(X, P, sl, 0, j, r);
            float2 *R0 = X + (60 + 4 * (j & 7)) * P + sl.own;
            R0[0] = r.rho;
            R0[P] = r.mx;
            R0[2 * P] = r.my;
            R0[3 * P] = r.E;
        }
        if (j >= 3 && j <= R + 6) march_publish(X, P, sl, 1, j, b_p1);
        if (j >= 6 && j <= R + 7) march_publish(X, P, sl, 2, j, c_p1);
        __syncthreads();
        if (j + 1 <= R + 5) load_row(j + 1);

        if (j >= 8 && j <= R + 5) {
            // steady state: the three stages without branches between them, so
            // that the compiler interleaves their independent arithmetic (with
            // one or two CTAs per SM the latency is hidden by this ILP)
            float2 L3[4], L2[4], L1[4];
            march_rhs<true>(X, P, nb, 2, j, c_m1, c_c, c_p1, u.inv_h, u.inv_2h, mu, kap, yf3, L3);
            march_rhs<true>(X, P, nb, 1, j, b_m1, b_c, b_p1, u.inv_h, u.inv_2h, mu, kap, yf2, L2);
            march_rhs<true>(X, P, nb, 0, j, a_m1, a_c, a_p1, u.inv_h, u.inv_2h, mu, kap, yf1, L1);
            {
                const float2 *R0 = X + (60 + 4 * ((j - 5) & 7)) * P + sl.own;
                const float2 q[4] = {c_c.rho, c_c.mx, c_c.my, c_c.E};
                float *o = u.out + wrap_index(u.y0 - 8 + j, n) * n;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 base = R0[k * P];
                    const float2 res = fma2(f2(2.f / 3.f), add2(sub2(q[k], base), mul2(dt, L3[k])), base);
                    if (wa) o[k * plane + xa] = res.x;
                    if (wb) o[k * plane + xb] = res.y;
                }
            }
            {
                const float2 *R0 = X + (60 + 4 * ((j - 3) & 7)) * P + sl.own;
                const float2 q[4] = {b_c.rho, b_c.mx, b_c.my, b_c.E};
                float2 sv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 base = R0[k * P];
                    sv[k] = fma2(f2(0.25f), add2(sub2(q[k], base), mul2(dt, L2[k])), base);
                }
                c_m1 = c_c;
                c_c = c_p1;
                c_p1 = make_rec(sv[0], sv[1], sv[2], sv[3], gm1);
            }
            {
                const float2 q[4] = {a_c.rho, a_c.mx, a_c.my, a_c.E};
                float2 sv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) sv[k] = add2(q[k], mul2(dt, L1[k]));
                b_m1 = b_c;
                b_c = b_p1;
                b_p1 = make_rec(sv[0], sv[1], sv[2], sv[3], gm1);
            }
            continue;
        }
        // stage 3 at row y0 - 8 + j: the new state
        if (j == 7) march_rhs<false>(X, P, nb, 2, j, c_m1, c_c, c_p1, u.inv_h, u.inv_2h, mu, kap, yf3, L);
        if (j >= 8) {
            march_rhs<true>(X, P, nb, 2, j, c_m1, c_c, c_p1, u.inv_h, u.inv_2h, mu, kap, yf3, L);
            const float2 *R0 = X + (60 + 4 * ((j - 5) & 7)) * P + sl.own;
            const float2 q[4] = {c_c.rho, c_c.mx, c_c.my, c_c.E};
            float *o = u.out + wrap_index(u.y0 - 8 + j, n) * n;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 base = R0[k * P];
                const float2 res = fma2(f2(2.f / 3.f), add2(sub2(q[k], base), mul2(dt, L[k])), base);
                if (wa) o[k * plane + xa] = res.x;
                if (wb) o[k * plane + xb] = res.y;
            }
        }
        // stage 2 at row y0 - 6 + j
        if (j == 4) march_rhs<false>(X, P, nb, 1, j, b_m1, b_c, b_p1, u.inv_h, u.inv_2h, mu, kap, yf2, L);
        if (j >= 5 && j <= R + 6) {
            march_rhs<true>(X, P, nb, 1, j, b_m1, b_c, b_p1, u.inv_h, u.inv_2h, mu, kap, yf2, L);
            const float2 *R0 = X + (60 + 4 * ((j - 3) & 7)) * P + sl.own;
            const float2 q[4] = {b_c.rho, b_c.mx, b_c.my, b_c.E};
            float2 s[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 base = R0[k * P];
                s[k] = fma2(f2(0.25f), add2(sub2(q[k], base), mul2(dt, L[k])), base);
            }
            c_m1 = c_c;
            c_c = c_p1;
            c_p1 = make_rec(s[0], s[1], s[2], s[3], gm1);
        }
        // stage 1 at row y0 - 4 + j
        if (j == 1) march_rhs<false>(X, P, nb, 0, j, a_m1, a_c, a_p1, u.inv_h, u.inv_2h, mu, kap, yf1, L);
        if (j >= 2 && j <= R + 5) {
            march_rhs<true>(X, P, nb, 0, j, a_m1, a_c, a_p1, u.inv_h, u.inv_2h, mu, kap, yf1, L);
            const float2 q[4] = {a_c.rho, a_c.mx, a_c.my, a_c.E};
            float2 s[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] = add2(q[k], mul2(dt, L[k]));
            b_m1 = b_c;
            b_c = b_p1;
            b_p1 = make_rec(s[0], s[1], s[2], s[3], gm1);
        }
    }
}

// After an odd number of steps the states sit in the scratch buffers: copy
// them back (group blockIdx.y).
template <class Units>
__global__ void __launch_bounds__(256) ns2d_copy_back(Units src) {
    const NsGroup<float> G = src.group(blockIdx.y);
    const size_t count = (size_t)G.n * G.n * G.nprob;  // float4 per group: 4 n^2 nprob floats
    const float4 *s = reinterpret_cast<const float4 *>(G.s1);
    float4 *d = reinterpret_cast<float4 *>(G.u0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

// CTAs per launch of the persistent step kernel: resident CTAs per SM x SMs
// (per device: the attribute and the occupancy belong to a device context)
template <int TX, int H, int MINB, class Tiles>
static int step_grid(int total_tiles) {
    static OncePerDevice once;
    static int ctas[kMaxDevices];
    once.run([](int dev) {
        const size_t smem = StepSmem<TX, H>::bytes();
        int per_sm = 0, sms = 0;
        cudaError_t e = cudaFuncSetAttribute(ns2d_rk3_step<TX, H, MINB, Tiles>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ns2d_rk3_step<TX, H, MINB, Tiles>, 256, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ctas[dev] = std::max(per_sm, 1) * std::max(sms, 1);
        return e;
    });
    const int dev = OncePerDevice::current();
    const int c = dev >= 0 && ctas[dev] > 0 ? ctas[dev] : kNumSMs;
    return std::min(total_tiles, c);
}

template <int TX, int H, int MINB, class Tiles>
static void step_launch(const Tiles &src, int total_tiles, int parity, float gm1, float mu, float kap,
                        cudaStream_t s) {
    const int grid = step_grid<TX, H, MINB, Tiles>(total_tiles);
    // programmatic stream serialisation: the launch may start while the
    // previous kernel on the stream finishes; the kernel waits for it before
    // it touches the state (griddepcontrol.wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = StepSmem<TX, H>::bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, ns2d_rk3_step<TX, H, MINB, Tiles>, src, total_tiles, parity, gm1, mu, kap);
}

// nsteps steps of every tile (the states end in u0), FP32
template <int TX, int H, int MINB, class Tiles>
static void step_sequence(const Tiles &src, int ngroups, int total_tiles, int nsteps, float gm1, float mu,
                          float kap, cudaStream_t s) {
    for (int st = 0; st < nsteps; ++st) step_launch<TX, H, MINB>(src, total_tiles, st & 1, gm1, mu, kap, s);
    count_launches(nsteps);
    if (nsteps & 1) {
        ns2d_copy_back<Tiles><<<dim3(2 * kNumSMs, ngroups), 256, 0, s>>>(src);
        count_launches(1);
    }
}

template <class Units>
static void march_launch(const Units &src, int units, int threads, int parity, float gm1, float mu, float kap,
                         cudaStream_t s) {
    static OncePerDevice once;
    once.run([](int) {
        return cudaFuncSetAttribute(ns2d_rk3_march<Units>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)march_smem_bytes(kMarchMaxThreads));
    });
    // programmatic stream serialisation: the launch may start while the
    // previous kernel on the stream finishes; the kernel waits for it before
    // it touches the state (griddepcontrol.wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(units);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = march_smem_bytes(threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, ns2d_rk3_march<Units>, src, parity, gm1, mu, kap);
}

// nsteps steps of every unit (the states end in u0), FP32
template <class Units>
static void march_sequence(const Units &src, int ngroups, int units, int threads, int nsteps, float gm1, float mu,
                           float kap, cudaStream_t s) {
    for (int st = 0; st < nsteps; ++st) march_launch(src, units, threads, st & 1, gm1, mu, kap, s);
    count_launches(nsteps);
    if (nsteps & 1) {
        ns2d_copy_back<Units><<<dim3(2 * kNumSMs, ngroups), 256, 0, s>>>(src);
        count_launches(1);
    }
}

// rows per segment of the march for a choice (the batch's tuned "shape":
// shape mod kNsSegChoices the segment rows, shape / kNsSegChoices = 1 narrow
// bands)
int ns2d_seg_rows(int shape) {
    constexpr int rows[kNsSegChoices] = {32, 16, 64, 128, 256, 24, 48, 20};
    return rows[shape % kNsSegChoices];
}
bool ns2d_narrow(int shape) { return shape / kNsSegChoices == 1; }

int ns2d_default_choice(int n, int grids, int sms) {
    const int base = n > 256 ? kNsSegChoices : 0;
    constexpr int longest_first[kNsSegChoices] = {4, 3, 2, 6, 0, 5, 7, 1};  // 256, 128, 64, 48, 32, 24, 20, 16 rows
    for (int r : longest_first) {
        int bands = 0, segs = 0, threads = 0;
        ns2d_march_layout(n, base + r, &bands, &segs, &threads);
        if ((long long)bands * segs * grids >= 2LL * sms) return base + r;
    }
    return base + 1;
}

void ns2d_march_layout(int n, int shape, int *bands, int *segs, int *threads) {
    const int S = std::min(n, ns2d_seg_rows(shape));
    const bool narrow = ns2d_narrow(shape);
    *bands = march_bands(n, narrow);
    *segs = (n + S - 1) / S;
    *threads = march_threads(n, narrow);
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
        // the copy back moves float4
        if ((reinterpret_cast<uintptr_t>(whole) | reinterpret_cast<uintptr_t>(split) |
             reinterpret_cast<uintptr_t>(scratch)) & 15)
            return cudaErrorMisalignedAddress;
        if (n_split_probs > 0) {
            // a handle (members and fine run): both groups in one persistent
            // launch of the tile kernel per step
            PairTiles P{{A.g[0], A.g[1]}};
            P.g[0].tile_begin = 0;
            P.g[1].tile_begin = tiles[0];
            step_sequence<32, 16, 2>(P, 2, grid, nsteps, A.gm1, A.mu, A.kappa, stream);
        } else {
            // grids of one size (truth runs, the stateless entry point): the
            // column march
            OneUnits U{A.g[0]};
            int bands = 0, segs = 0, threads = 0;
            ns2d_march_layout(ns[0], np[0] == 1 ? 1 : 0, &bands, &segs, &threads);
            U.g.tx = bands;
            U.g.ty = segs;
            U.g.tile_begin = 0;
            march_sequence(U, 1, bands * segs * np[0], threads, nsteps, A.gm1, A.mu, A.kappa, stream);
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

static cudaError_t table_steps(const NsGroup<float> *d_groups, int ngroups, int units, int n, int nsteps,
                               bool probe, double gamma, double mu, double prandtl, int shape, cudaStream_t s) {
    if (units == 0 || nsteps == 0) return cudaSuccess;
    const float gm1 = (float)(gamma - 1.0), m = (float)mu, kap = (float)(mu * gamma / ((gamma - 1.0) * prandtl));
    const TableUnits src{d_groups, ngroups};
    const int threads = march_threads(n, ns2d_narrow(shape));
    if (probe) {  // one step into the scratch buffers: the states stay as they are
        march_launch(src, units, threads, 0, gm1, m, kap, s);
        count_launches(1);
    } else {
        march_sequence(src, ngroups, units, threads, nsteps, gm1, m, kap, s);
    }
    return cudaGetLastError();
}

cudaError_t ns2d_forecast_table(const NsGroup<float> *d_groups, int ngroups, int units, int n, int nsteps,
                                double gamma, double mu, double prandtl, int shape, cudaStream_t s) {
    return table_steps(d_groups, ngroups, units, n, nsteps, false, gamma, mu, prandtl, shape, s);
}

cudaError_t ns2d_probe_step(const NsGroup<float> *d_groups, int ngroups, int units, int n, double gamma,
                            double mu, double prandtl, int shape, cudaStream_t s) {
    return table_steps(d_groups, ngroups, units, n, 1, true, gamma, mu, prandtl, shape, s);
}

#define MGK_NS_INST(T)                                                                            \
    template cudaError_t ns2d_forecast<T>(T *, int, int, T *, int, int, double, double, double,    \
                                          double, double, int, cudaStream_t);                     \
    template cudaError_t ns2d_forecast_scratch<T>(T *, int, int, T *, int, int, double, double,    \
                                                  double, double, double, int, T *, cudaStream_t);

MGK_NS_INST(float)
MGK_NS_INST(double)
#undef MGK_NS_INST

}  // namespace mgk
