// lbm_q27.cu -- single-phase D3Q27 step (App. D of arXiv:2010.01628), central
// moments and the raw-moment variant, FP64 or FP32 storage of f - w.
//
// The App. D basis is spanned by the monomials cbar_x^a cbar_y^b cbar_z^c
// (a, b, c <= 2) and the lattice is the tensor product of three D1Q3 lattices,
// so the whole back-transform f* = M^-1 N^-1 k* factorises into 1D transforms
// along z, y and x (each: binomial shift of three central moments to raw
// moments by u_a, then D1Q3 populations).  The collision needs from the
// populations only rho, j and the six raw second moments: every central moment
// except the five deviatoric second-order ones is set by rho and F (the
// Galilean-invariant equilibrium and the central-Hermite force term of App. B).
//
// Deviation form (FP32 accuracy near rho = 1): with E the central moments of
// the rest state (rho = 1, u = 0), f* - w = T1D(u)[k* - E] + (prod phi(u) - prod w),
// where phi(u) = ((c_s^2 + u^2 - u)/2, 1 - c_s^2 - u^2, (c_s^2 + u^2 + u)/2)
// is the D1Q3 equilibrium of unit density; the product difference is formed
// term by term (d_x b c + A (d_y c + B d_z)), so nothing cancels.  The
// raw-moment variant works the same way with no shift (T1D(0)) and raw
// equilibrium moments rho prod(1, u, u^2 + c_s^2).
#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace lbm {
namespace q27 {

// App. D lattice order; opposite(i) = i +/- 13.
__host__ __device__ constexpr int cx(int i) {
    constexpr int t[27] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, -1, -1, -1, -1, 1, 0, 0, 1, 1, 1, 1, 0, 0, 1, 1, 1, 1};
    return t[i];
}
__host__ __device__ constexpr int cy(int i) {
    constexpr int t[27] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, -1, -1, 1, 1, 0, 1, 0, 1, -1, 0, 0, 1, 1, 1, 1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int cz(int i) {
    constexpr int t[27] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 13 ? i + 13 : i - 13); }
__host__ __device__ constexpr double w1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double w(int i) { return w1(cx(i)) * w1(cy(i)) * w1(cz(i)); }

struct Args {
    Box box;
    double omega;
    double g[3];
    double lid[3];
};

template <typename S, typename C, int I>
__device__ __forceinline__ C load_dev(const S* p) {
    return (C)Store<S>::load(p);
}

// One pulled population f_I(x) = f*_I(x - c_I) (shifted), half-way bounce-back
// with Ladd's moving-lid term 6 w_I c_I . u_lid beyond the +y face.
template <typename S, typename C, bool WALLS, int I>
__device__ __forceinline__ C gather_one(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y, int z,
                                        uint32_t self, const Args& p) {
    constexpr int ex = cx(I), ey = cy(I), ez = cz(I);
    const int sx = ex == 0 ? x : (ex > 0 ? q.xm : q.xp);
    const int sy = ey == 0 ? y : (ey > 0 ? q.ym : q.yp);
    const int sz = ez == 0 ? z : (ez > 0 ? q.zm : q.zp);
    const bool wall = WALLS && ((ex > 0 && q.wxm) || (ex < 0 && q.wxp) || (ey > 0 && q.wym) || (ey < 0 && q.wyp) ||
                                (ez > 0 && q.wzm) || (ez < 0 && q.wzp));
    if (!wall) {
        const uint32_t cell = ((uint32_t)sz * (uint32_t)b.ny + (uint32_t)sy) * (uint32_t)b.nx + (uint32_t)sx;
        return load_dev<S, C, I>(src + (size_t)I * b.n + cell);
    }
    C v = load_dev<S, C, opp(I)>(src + (size_t)opp(I) * b.n + self);
    if (ey < 0 && q.wyp)
        v += (C)(6.0 * w(I)) * ((C)ex * (C)p.lid[0] + (C)ey * (C)p.lid[1] + (C)ez * (C)p.lid[2]);
    return v;
}

// Populations in a cube g[cx+1][cy+1][cz+1].
template <typename S, typename C, bool WALLS>
__device__ __forceinline__ void gather(const S* __restrict__ src, const Box& b, const Nbr& q, int x, int y, int z,
                                       uint32_t self, const Args& p, C (&g)[3][3][3]) {
#define Q27_G(I) g[cx(I) + 1][cy(I) + 1][cz(I) + 1] = gather_one<S, C, WALLS, I>(src, b, q, x, y, z, self, p);
    Q27_G(0) Q27_G(1) Q27_G(2) Q27_G(3) Q27_G(4) Q27_G(5) Q27_G(6) Q27_G(7) Q27_G(8) Q27_G(9) Q27_G(10) Q27_G(11)
    Q27_G(12) Q27_G(13) Q27_G(14) Q27_G(15) Q27_G(16) Q27_G(17) Q27_G(18) Q27_G(19) Q27_G(20) Q27_G(21) Q27_G(22)
    Q27_G(23) Q27_G(24) Q27_G(25) Q27_G(26)
#undef Q27_G
}

template <typename S, typename C>
__device__ __forceinline__ void scatter(S* __restrict__ dst, size_t n, uint32_t self, const C (&g)[3][3][3]) {
#define Q27_S(I) Store<S>::store(dst + (size_t)I * n + self, g[cx(I) + 1][cy(I) + 1][cz(I) + 1]);
    Q27_S(0) Q27_S(1) Q27_S(2) Q27_S(3) Q27_S(4) Q27_S(5) Q27_S(6) Q27_S(7) Q27_S(8) Q27_S(9) Q27_S(10) Q27_S(11)
    Q27_S(12) Q27_S(13) Q27_S(14) Q27_S(15) Q27_S(16) Q27_S(17) Q27_S(18) Q27_S(19) Q27_S(20) Q27_S(21) Q27_S(22)
    Q27_S(23) Q27_S(24) Q27_S(25) Q27_S(26)
#undef Q27_S
}

// rho - 1, j and the raw second moments of the shifted populations (the rest
// state's parts: none for j and the off-diagonal moments; c_s^2 on each
// diagonal one, which cancels in the deviatoric differences).
template <typename C>
struct Mom {
    C drho, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz;
};

template <typename C>
__device__ __forceinline__ Mom<C> moments(const C (&g)[3][3][3]) {
    // x-lines first: s[b][c] = sum, d[b][c] = f(+1) - f(-1), e[b][c] = f(+1) + f(-1)
    C s[3][3], d[3][3], e[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e[b][c] = g[2][b][c] + g[0][b][c];
            d[b][c] = g[2][b][c] - g[0][b][c];
            s[b][c] = e[b][c] + g[1][b][c];
        }
    Mom<C> m;
    C S = (C)0, X = (C)0, XX = (C)0, Y = (C)0, YY = (C)0, Z = (C)0, ZZ = (C)0, XY = (C)0, XZ = (C)0, YZ = (C)0;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int ey = b - 1, ez = c - 1;
            S += s[b][c];
            X += d[b][c];
            XX += e[b][c];
            if (ey) {
                Y += (C)ey * s[b][c];
                YY += s[b][c];
                XY += (C)ey * d[b][c];
            }
            if (ez) {
                Z += (C)ez * s[b][c];
                ZZ += s[b][c];
                XZ += (C)ez * d[b][c];
            }
            if (ey * ez) YZ += (C)(ey * ez) * s[b][c];
        }
    m.drho = S;
    m.jx = X;
    m.jy = Y;
    m.jz = Z;
    m.pxx = XX;
    m.pyy = YY;
    m.pzz = ZZ;
    m.pxy = XY;
    m.pxz = XZ;
    m.pyz = YZ;
    return m;
}

// One line: three moments (orders 0..2) about u -> raw moments -> D1Q3.
template <typename C>
__device__ __forceinline__ void line(C& a0, C& a1, C& a2, C u) {
    const C r1 = a1 + u * a0;
    const C r2 = a2 + u * ((C)2 * a1 + u * a0);
    const C r0 = a0;
    a0 = (C)0.5 * (r2 - r1);
    a1 = r0 - r2;
    a2 = (C)0.5 * (r2 + r1);
}

// Moments k[a][b][c] -> populations [cx+1][cy+1][cz+1], sweeping z, y, x.
template <typename C>
__device__ __forceinline__ void to_populations(C (&k)[3][3][3], C ux, C uy, C uz) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) line<C>(k[a][b][0], k[a][b][1], k[a][b][2], uz);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) line<C>(k[a][0][c], k[a][1][c], k[a][2][c], uy);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) line<C>(k[0][b][c], k[1][b][c], k[2][b][c], ux);
}

struct Rest {  // central moments of the rest state per axis: (1, 0, c_s^2)
    __host__ __device__ static constexpr double m(int a) { return a == 0 ? 1.0 : (a == 1 ? 0.0 : 1.0 / 3.0); }
};

// Central force moments R[a][b][c] = F_x a m(a-1) m(b) m(c) + ... (App. B).
template <typename C>
__device__ __forceinline__ C force_moment(int a, int b, int c, C Fx, C Fy, C Fz) {
    C v = (C)0;
    if (a >= 1) v += Fx * (C)(a * Rest::m(a - 1) * Rest::m(b) * Rest::m(c));
    if (b >= 1) v += Fy * (C)(b * Rest::m(a) * Rest::m(b - 1) * Rest::m(c));
    if (c >= 1) v += Fz * (C)(c * Rest::m(a) * Rest::m(b) * Rest::m(c - 1));
    return v;
}

// f* - w of the central-moment collision (deviation form).
template <typename C>
__device__ __forceinline__ void collide_cm(C (&g)[3][3][3], const Mom<C>& m, C rho, C ux, C uy, C uz, C Fx, C Fy,
                                           C Fz, C omega) {
    const C om1 = (C)1 - omega;
    // deviatoric central second moments: raw minus rho u u plus (u F + F u)/2
    const C d1 = om1 * ((m.pxx - m.pyy) - rho * (ux * ux - uy * uy) + (ux * Fx - uy * Fy));
    const C d2 = om1 * ((m.pxx - m.pzz) - rho * (ux * ux - uz * uz) + (ux * Fx - uz * Fz));
    const C kxy = om1 * (m.pxy - rho * ux * uy + (C)0.5 * (ux * Fy + uy * Fx));
    const C kxz = om1 * (m.pxz - rho * ux * uz + (C)0.5 * (ux * Fz + uz * Fx));
    const C kyz = om1 * (m.pyz - rho * uy * uz + (C)0.5 * (uy * Fz + uz * Fy));
    const C drho = m.drho;
    // k* - E: equilibrated moments rho prod m + R/2 minus the rest moments prod m
    C k[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                k[a][b][c] = drho * (C)(Rest::m(a) * Rest::m(b) * Rest::m(c)) + (C)0.5 * force_moment<C>(a, b, c, Fx, Fy, Fz);
    const C third = (C)(1.0 / 3.0);
    k[2][0][0] = (drho + d1 + d2) * third;
    k[0][2][0] = (drho - (C)2 * d1 + d2) * third;
    k[0][0][2] = (drho + d1 - (C)2 * d2) * third;
    k[1][1][0] = kxy;
    k[1][0][1] = kxz;
    k[0][1][1] = kyz;
    to_populations<C>(k, ux, uy, uz);
    // + (prod phi(u) - prod w), d = phi - w per axis
    const C cs2 = (C)(1.0 / 3.0);
    C ph[3][3], dl[3][3];  // [axis][c + 1]
    const C uu[3] = {ux, uy, uz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const C u = uu[ax], u2 = u * u;
        dl[ax][0] = (C)0.5 * (u2 - u);
        dl[ax][1] = -u2;
        dl[ax][2] = (C)0.5 * (u2 + u);
        ph[ax][0] = (C)0.5 * cs2 + dl[ax][0];
        ph[ax][1] = (C)1 - cs2 + dl[ax][1];
        ph[ax][2] = (C)0.5 * cs2 + dl[ax][2];
    }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const C pp = ph[1][b] * ph[2][c];
            const C qq = dl[1][b] * ph[2][c] + (C)w1(b - 1) * dl[2][c];
#pragma unroll
            for (int a = 0; a < 3; ++a) g[a][b][c] = k[a][b][c] + dl[0][a] * pp + (C)w1(a - 1) * qq;
        }
}

// f* - w of the raw-moment variant (T = M): raw equilibrium rho prod(1, u, u^2 + c_s^2),
// the force term's raw moments (its central ones shifted by u), the same K.
template <typename C>
__device__ __forceinline__ void collide_rm(C (&g)[3][3][3], const Mom<C>& m, C rho, C ux, C uy, C uz, C Fx, C Fy,
                                           C Fz, C omega) {
    const C om1 = (C)1 - omega, oh = (C)1 - (C)0.5 * omega;
    const C drho = m.drho;
    // force: central moments, then shifted along x, y, z to raw moments
    C R[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) R[a][b][c] = force_moment<C>(a, b, c, Fx, Fy, Fz);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R[2][b][c] += ux * ((C)2 * R[1][b][c] + ux * R[0][b][c]);
            R[1][b][c] += ux * R[0][b][c];
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R[a][2][c] += uy * ((C)2 * R[a][1][c] + uy * R[a][0][c]);
            R[a][1][c] += uy * R[a][0][c];
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            R[a][b][2] += uz * ((C)2 * R[a][b][1] + uz * R[a][b][0]);
            R[a][b][1] += uz * R[a][b][0];
        }
    // raw equilibrium minus the rest moments: rho prod mr - prod m, mr = m + d, d = (0, u, u^2)
    const C uu[3] = {ux, uy, uz};
    C mr[3][3], dm[3][3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        dm[ax][0] = (C)0;
        dm[ax][1] = uu[ax];
        dm[ax][2] = uu[ax] * uu[ax];
        mr[ax][0] = (C)1;
        mr[ax][1] = uu[ax];
        mr[ax][2] = (C)(1.0 / 3.0) + dm[ax][2];
    }
    C k[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const C pd = dm[0][a] * mr[1][b] * mr[2][c] +
                             (C)Rest::m(a) * (dm[1][b] * mr[2][c] + (C)Rest::m(b) * dm[2][c]);
                k[a][b][c] = rho * pd + drho * (C)(Rest::m(a) * Rest::m(b) * Rest::m(c)) + (C)0.5 * R[a][b][c];
            }
    // second order: trace at equilibrium, deviatoric and off-diagonal relaxed
    const C exx = rho * dm[0][2], eyy = rho * dm[1][2], ezz = rho * dm[2][2];  // minus the rest c_s^2 (rho - 1 below)
    const C d1 = om1 * (m.pxx - m.pyy) + omega * (exx - eyy) + oh * (R[2][0][0] - R[0][2][0]);
    const C d2 = om1 * (m.pxx - m.pzz) + omega * (exx - ezz) + oh * (R[2][0][0] - R[0][0][2]);
    const C tr = drho + exx + eyy + ezz + (C)0.5 * (R[2][0][0] + R[0][2][0] + R[0][0][2]);
    const C third = (C)(1.0 / 3.0);
    k[2][0][0] = (tr + d1 + d2) * third;
    k[0][2][0] = (tr - (C)2 * d1 + d2) * third;
    k[0][0][2] = (tr + d1 - (C)2 * d2) * third;
    k[1][1][0] = om1 * m.pxy + omega * rho * ux * uy + oh * R[1][1][0];
    k[1][0][1] = om1 * m.pxz + omega * rho * ux * uz + oh * R[1][0][1];
    k[0][1][1] = om1 * m.pyz + omega * rho * uy * uz + oh * R[0][1][1];
    to_populations<C>(k, (C)0, (C)0, (C)0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) g[a][b][c] = k[a][b][c];
}

template <typename C>
struct Node {
    C rho, ux, uy, uz, Fx, Fy, Fz;
};

template <typename C>
__device__ __forceinline__ Node<C> macro(const Mom<C>& m, const Args& p) {
    Node<C> s;
    s.rho = (C)1 + m.drho;
    s.Fx = s.rho * (C)p.g[0];
    s.Fy = s.rho * (C)p.g[1];
    s.Fz = s.rho * (C)p.g[2];
    const C inv = recip(s.rho);
    s.ux = (m.jx + (C)0.5 * s.Fx) * inv;
    s.uy = (m.jy + (C)0.5 * s.Fy) * inv;
    s.uz = (m.jz + (C)0.5 * s.Fz) * inv;
    return s;
}

template <typename S, typename C, bool WALLS, bool RM>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ src, S* __restrict__ dst, Args p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx) return;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C g[3][3][3];
    gather<S, C, WALLS>(src, b, q, x, y, z, self, p, g);
    const Mom<C> m = moments<C>(g);
    const Node<C> s = macro<C>(m, p);
    if (RM)
        collide_rm<C>(g, m, s.rho, s.ux, s.uy, s.uz, s.Fx, s.Fy, s.Fz, (C)p.omega);
    else
        collide_cm<C>(g, m, s.rho, s.ux, s.uy, s.uz, s.Fx, s.Fy, s.Fz, (C)p.omega);
    scatter<S, C>(dst, b.n, self, g);
}

// f - w = rho (prod phi(u) - prod w) + (rho - 1) w.
template <typename S, typename C>
__global__ void init_kernel(S* __restrict__ dst, const double* __restrict__ slab, Box b, int z0, int nzs, bool uniform) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    if (x >= b.nx || zs >= nzs) return;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)(z0 + zs) * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    double rho = 1.0, u[3] = {0.0, 0.0, 0.0};
    if (!uniform) {
        rho = slab[k];
        u[0] = slab[m + k];
        u[1] = slab[2 * m + k];
        u[2] = slab[3 * m + k];
    }
    const double drho = uniform ? 0.0 : slab[k] - 1.0;
    double ph[3][3], dl[3][3];
    for (int ax = 0; ax < 3; ++ax) {
        const double v = u[ax], v2 = v * v;
        dl[ax][0] = 0.5 * (v2 - v);
        dl[ax][1] = -v2;
        dl[ax][2] = 0.5 * (v2 + v);
        ph[ax][0] = 1.0 / 6.0 + dl[ax][0];
        ph[ax][1] = 2.0 / 3.0 + dl[ax][1];
        ph[ax][2] = 1.0 / 6.0 + dl[ax][2];
    }
    C g[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double pd = dl[0][a] * ph[1][bb] * ph[2][c] +
                                  w1(a - 1) * (dl[1][bb] * ph[2][c] + w1(bb - 1) * dl[2][c]);
                g[a][bb][c] = (C)(rho * pd + drho * w1(a - 1) * w1(bb - 1) * w1(c - 1));
            }
    scatter<S, C>(dst, b.n, self, g);
}

template <typename S, typename C, bool WALLS>
__global__ void fields_kernel(const S* __restrict__ src, double* __restrict__ slab, Args p, int z0, int nzs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, zs = blockIdx.z;
    const Box& b = p.box;
    if (x >= b.nx || zs >= nzs) return;
    const int z = z0 + zs;
    const size_t m = (size_t)b.nx * b.ny * nzs;
    const size_t k = ((size_t)zs * b.ny + y) * b.nx + x;
    const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
    const Nbr q = make_nbr(b, x, y, z);
    C g[3][3][3];
    gather<S, C, WALLS>(src, b, q, x, y, z, self, p, g);
    const Node<C> s = macro<C>(moments<C>(g), p);
    slab[k] = (double)s.rho;
    slab[m + k] = (double)s.ux;
    slab[2 * m + k] = (double)s.uy;
    slab[3 * m + k] = (double)s.uz;
}

template <typename S, typename C, bool WALLS>
__global__ void __launch_bounds__(RED_THREADS) reduce_kernel(const S* __restrict__ src, Args p, C* __restrict__ uprev,
                                                             bool have_prev, bool record, double* __restrict__ partials) {
    const Box& b = p.box;
    const int chunks_x = (b.nx + RED_THREADS - 1) / RED_THREADS;
    const long total = (long)chunks_x * b.ny * b.nz;
    RedAcc acc;
    acc.zero();
    for (long ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int cxk = (int)(ch % chunks_x);
        const long row = ch / chunks_x;
        const int y = (int)(row % b.ny), z = (int)(row / b.ny);
        const int x = cxk * RED_THREADS + threadIdx.x;
        if (x < b.nx) {
            const uint32_t self = ((uint32_t)z * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nx + (uint32_t)x;
            const Nbr q = make_nbr(b, x, y, z);
            C g[3][3][3];
            gather<S, C, WALLS>(src, b, q, x, y, z, self, p, g);
            const Node<C> s = macro<C>(moments<C>(g), p);
            reduce_node<C>(acc, s.rho, s.ux, s.uy, s.uz, uprev, b.n, self, have_prev, record);
        }
    }
    block_reduce_store(acc, partials);
}

static Args args_of(const lbm_ctx* c) {
    Args p;
    p.box = c->box;
    p.omega = c->relax.omega;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = c->forcing.g[a];
        p.lid[a] = (c->box.periodic & 2u) ? 0.0 : c->grid.lid_u[a];
    }
    return p;
}

template <typename S, typename C>
static cudaError_t step_t(lbm_ctx* c, long n, bool dry) {
    const Args p = args_of(c);
    const bool walls = (c->box.periodic & 7u) != 7u, rm = c->relax.moment_space == LBM_MOMENTS_RAW;
    const int bx = c->block_x;
    const dim3 grid = step_grid(c->box, bx);
    for (long s = 0; s < n; ++s) {
        const S* src = (const S*)c->buf[c->cur];
        S* dst = (S*)c->buf[c->cur ^ 1];
        if (walls)
            rm ? step_kernel<S, C, true, true><<<grid, bx, 0, c->stream>>>(src, dst, p)
               : step_kernel<S, C, true, false><<<grid, bx, 0, c->stream>>>(src, dst, p);
        else
            rm ? step_kernel<S, C, false, true><<<grid, bx, 0, c->stream>>>(src, dst, p)
               : step_kernel<S, C, false, false><<<grid, bx, 0, c->stream>>>(src, dst, p);
        if (!dry) c->cur ^= 1;
    }
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t init_t(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    init_kernel<S, C><<<grid, bx, 0, c->stream>>>((S*)c->buf[c->cur], slab, c->box, z0, nzs, uniform);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t fields_t(lbm_ctx* c, double* slab, int z0, int nzs) {
    const Args p = args_of(c);
    const int bx = c->block_x;
    dim3 grid((unsigned)((c->box.nx + bx - 1) / bx), (unsigned)c->box.ny, (unsigned)nzs);
    if ((c->box.periodic & 7u) != 7u)
        fields_kernel<S, C, true><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    else
        fields_kernel<S, C, false><<<grid, bx, 0, c->stream>>>((const S*)c->buf[c->cur], slab, p, z0, nzs);
    return cudaGetLastError();
}

template <typename S, typename C>
static cudaError_t reduce_t(lbm_ctx* c, bool record) {
    const Args p = args_of(c);
    if ((c->box.periodic & 7u) != 7u)
        reduce_kernel<S, C, true><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>((const S*)c->buf[c->cur], p, (C*)c->uprev,
                                                                             c->have_prev, record, c->partials);
    else
        reduce_kernel<S, C, false><<<RED_BLOCKS, RED_THREADS, 0, c->stream>>>(
            (const S*)c->buf[c->cur], p, (C*)c->uprev, c->have_prev, record, c->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_finalize(c);
}

}  // namespace q27

cudaError_t q27_step(lbm_ctx* c, long n, bool dry) {
    return c->prec == LBM_FP64 ? q27::step_t<double, double>(c, n, dry) : q27::step_t<float, float>(c, n, dry);
}
cudaError_t q27_init(lbm_ctx* c, const double* slab, int z0, int nzs, bool uniform) {
    return c->prec == LBM_FP64 ? q27::init_t<double, double>(c, slab, z0, nzs, uniform)
                               : q27::init_t<float, float>(c, slab, z0, nzs, uniform);
}
cudaError_t q27_fields(lbm_ctx* c, double* slab, int z0, int nzs) {
    return c->prec == LBM_FP64 ? q27::fields_t<double, double>(c, slab, z0, nzs)
                               : q27::fields_t<float, float>(c, slab, z0, nzs);
}
cudaError_t q27_reduce(lbm_ctx* c, bool record) {
    return c->prec == LBM_FP64 ? q27::reduce_t<double, double>(c, record) : q27::reduce_t<float, float>(c, record);
}

}  // namespace lbm
