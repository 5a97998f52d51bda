// Fused field step + particle push of one tile (Sec. 1 of arXiv:2307.07999: the
// leapfrog of the Glasma links coupled to the CPIC push of the particles in them).
//
// The tile's links and phi (with a one-site halo) are already in shared memory
// for the field step, so the particles whose cell lies in the tile are pushed
// from there.  Their gather also needs the time-centred E on the link entering
// the cell from -x and from -y, i.e. E_{n+1/2} one site outside the tile; the
// CTA therefore also kicks E_x on the halo column x0-1 and E_y on the halo row
// y0-1 (not drifted, never stored to global memory).
#pragma once
#include "particles.cuh"

namespace glasma {

template <class T, int TX, int TY> struct FusedTile {
    static constexpr int HX = TX + 2, HS = HX * (TY + 2), FX = TX + 1, FS = FX * (TY + 1);
    static constexpr int SEX = (TX + 1) * TY;  // E_x average on x in [x0-1, x0+TX), y in tile
    static constexpr int SEY = TX * (TY + 1);  // E_y average on x in tile, y in [y0-1, y0+TY)
    static constexpr int SPI = TX * TY;        // pi average on the tile
    static constexpr size_t smem = sizeof(T) * (size_t)(2 * 18 * HS + 8 * HS + 8 * FS + 8 * (SEX + SEY + SPI));
};

// shared-memory field source for the push of the particles of one tile
template <class T, int TX, int TY> struct SmemSrc {
    static constexpr bool kRecord = false;
    using FT = FusedTile<T, TX, TY>;
    const T *sU, *sP, *sEx, *sEy, *sPi;
    int x0, y0, n;
    // offset of a (periodically wrapped) neighbour from the tile origin, in [-1, T]: the
    // tile's own cells keep their own slots even when the lattice is narrower than a tile
    DEV int hx(int x) const {
        int d = x - x0;
        if (d < -1) d += n;
        else if (d > TX) d -= n;
        return d + 1;
    }
    DEV int hy(int y) const {
        int d = y - y0;
        if (d < -1) d += n;
        else if (d > TY) d -= n;
        return d + 1;
    }
    // view of the fields around a cell of the tile: (dx, dy) offsets stay inside the halo
    struct View {
        const T *sU, *sP, *sEx, *sEy, *sPi;
        int hcx, hcy;  // the cell's slot coordinates in the halo tile
        DEV int h(int dx, int dy) const { return (hcy + dy) * FT::HX + hcx + dx; }
        DEV M3<T> link(int d, int dx, int dy) const { return sm_link<T, FT::HS>(sU, d, h(dx, dy)); }
        DEV void links(int dx, int dy, M3<T>& ux, M3<T>& uy) const {
            ux = link(0, dx, dy);
            uy = link(1, dx, dy);
        }
        DEV Al<T> phi(int dx, int dy) const { return sm_alg<T, FT::HS>(sP, h(dx, dy)); }
        DEV Al<T> eavg(int d, int dx, int dy) const {
            if (d == 0) return sm_alg<T, FT::SEX>(sEx, (hcy + dy - 1) * (TX + 1) + hcx + dx);
            return sm_alg<T, FT::SEY>(sEy, (hcy + dy) * TX + hcx + dx - 1);
        }
        DEV Al<T> piavg() const { return sm_alg<T, FT::SPI>(sPi, (hcy - 1) * TX + hcx - 1); }
    };
    DEV View view(int cx, int cy) const { return View{sU, sP, sEx, sEy, sPi, hx(cx), hy(cy)}; }
};

template <class T, int TX, int TY>
DEV void fused_tile(const StepArgs<T>& A, const PushArgs<T>& PA, int x0, int y0, const int* __restrict__ perm,
                    int ts, int tcount, unsigned char* smem_raw) {
    using FT = FusedTile<T, TX, TY>;
    constexpr int HX = FT::HX, HS = FT::HS, FX = FT::FX, FS = FT::FS;
    T* sU = reinterpret_cast<T*>(smem_raw);  // [2][18][HS]
    T* sP = sU + 2 * 18 * HS;                // [8][HS]
    T* sF = sP + 8 * HS;                     // [8][FS]
    T* sEx = sF + 8 * FS;                    // [8][SEX]
    T* sEy = sEx + 8 * FT::SEX;              // [8][SEY]
    T* sPi = sEy + 8 * FT::SEY;              // [8][SPI]
    const int n = A.n;
    const size_t ns = (size_t)n * n;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const T* __restrict__ src = A.src;
    const T dt = A.dtau, tb = A.tb, tp = A.tp, half = T(0.5);

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = (x < n) && (y < n);
    const size_t s = active ? (size_t)x + (size_t)n * y : 0;
    Al<T> Ex = load_alg(src, ns, P_EX, s), Ey = load_alg(src, ns, P_EY, s), pi = load_alg(src, ns, P_PI, s);

    // phase 1: links and phi of the tile and its halo
    for (int h = tid; h < HS; h += TX * TY) {
        const int hx = h % HX, hy = h / HX;
        const size_t g = (size_t)wrapi(x0 - 1 + hx, n) + (size_t)n * wrapi(y0 - 1 + hy, n);
        M3<T> UU[2];
        load_links(src, ns, g, UU[0], UU[1]);
#pragma unroll
        for (int d = 0; d < 2; d++) {
            const M3<T>& U = UU[d];
            T* b = sU + d * 18 * HS + h;
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    b[(2 * (3 * r + c)) * HS] = U.m[r][c].r;
                    b[(2 * (3 * r + c) + 1) * HS] = U.m[r][c].i;
                }
        }
        const Al<T> ph = load_alg(src, ns, P_PHI, g);
#pragma unroll
        for (int a = 0; a < 8; a++) sP[a * HS + h] = ph.a[a];
    }
    __syncthreads();
    // phase 2: ImTL P on [x0-1, x0+TX) x [y0-1, y0+TY)
    for (int i = tid; i < FS; i += TX * TY) {
        const int fx = i % FX, fy = i / FX;
        const int h = fy * HX + fx;
        const M3<T> a1 = mul(sm_link<T, HS>(sU, 0, h), sm_link<T, HS>(sU, 1, h + 1));
        const M3<T> b1 = mul(sm_link<T, HS>(sU, 1, h), sm_link<T, HS>(sU, 0, h + HX));
        const Al<T> F = im_tl(mul_nd(a1, b1));
#pragma unroll
        for (int a = 0; a < 8; a++) sF[a * FS + i] = F.a[a];
    }
    __syncthreads();

    // phase 3: kick and drift of the own site (as field_tile), keeping the E, pi averages
    if (active) {
        const int h = (threadIdx.y + 1) * HX + threadIdx.x + 1;
        const int f = (threadIdx.y + 1) * FX + threadIdx.x + 1;
        const Al<T> phi = sm_alg<T, HS>(sP, h);
        const M3<T> ux = sm_link<T, HS>(sU, 0, h), uy = sm_link<T, HS>(sU, 1, h);
        const M3<T> uxm = sm_link<T, HS>(sU, 0, h - 1), uym = sm_link<T, HS>(sU, 1, h - HX);
        const Al<T> psx = conj_alg(ux, sm_alg<T, HS>(sP, h + 1));
        const Al<T> psy = conj_alg(uy, sm_alg<T, HS>(sP, h + HX));
        Al<T> pin = pi;
        {
            const Al<T> chx = transport_alg(uxm, sm_alg<T, HS>(sP, h - 1));
            const Al<T> chy = transport_alg(uym, sm_alg<T, HS>(sP, h - HX));
#pragma unroll
            for (int a = 0; a < 8; a++)
                pin.a[a] += dt * tp * (psx.a[a] + chx.a[a] + psy.a[a] + chy.a[a] - T(4) * phi.a[a]);
        }
        const Al<T> F0 = sm_alg<T, FS>(sF, f);
        Al<T> Exn = Ex, Eyn = Ey;
        {
            const Al<T> cm = icomm(phi, psx);
            const Al<T> t1 = transport_alg(uym, sm_alg<T, FS>(sF, f - FX));
#pragma unroll
            for (int a = 0; a < 8; a++) Exn.a[a] += dt * (tb * (t1.a[a] - F0.a[a]) - tp * cm.a[a]);
        }
        {
            const Al<T> cm = icomm(phi, psy);
            const Al<T> t2 = transport_alg(uxm, sm_alg<T, FS>(sF, f - 1));
#pragma unroll
            for (int a = 0; a < 8; a++) Eyn.a[a] += dt * (tb * (F0.a[a] - t2.a[a]) - tp * cm.a[a]);
        }
        const int ex = threadIdx.y * (TX + 1) + threadIdx.x + 1, ey = (threadIdx.y + 1) * TX + threadIdx.x,
                  ep = threadIdx.y * TX + threadIdx.x;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            sEx[a * FT::SEX + ex] = half * (Ex.a[a] + Exn.a[a]);
            sEy[a * FT::SEY + ey] = half * (Ey.a[a] + Eyn.a[a]);
            sPi[a * FT::SPI + ep] = half * (pi.a[a] + pin.a[a]);
        }
        T* __restrict__ dst = A.dst;
        store_alg(dst, ns, P_EX, s, Exn);
        store_alg(dst, ns, P_EY, s, Eyn);
        store_alg(dst, ns, P_PI, s, pin);
        Al<T> phin;
#pragma unroll
        for (int a = 0; a < 8; a++) phin.a[a] = phi.a[a] + A.pe * pin.a[a];
        store_alg(dst, ns, P_PHI, s, phin);
        M3<T> Vn[2];
#pragma unroll
        for (int d = 0; d < 2; d++) {
            Al<T> e = d == 0 ? Exn : Eyn;
#pragma unroll
            for (int a = 0; a < 8; a++) e.a[a] *= A.ue;
            const M3<T> W = expi(herm(e));
            const M3<T>& U = d == 0 ? ux : uy;
            M3<T> V;
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    V.m[r][c] = val(cmac(cmac(cmul(W.m[r][0], U.m[0][c]), W.m[r][1], U.m[1][c]), W.m[r][2], U.m[2][c]));
            if (A.reunit == 1) reunit_rows(V);
            else if (A.reunit == 2 && sizeof(T) == 4) renorm_rows(V);
            Vn[d] = V;
        }
        store_links(dst, ns, s, Vn[0], Vn[1]);
    }
    const bool push = PA.acc != nullptr && tcount > 0;
    // phase 3b: E_x on the halo column and E_y on the halo row (kick only)
    if (push && tid < TX + TY) {
        const bool row = tid < TX;  // row: (x0 + tid, y0 - 1), E_y ; column: (x0 - 1, y0 + tid - TX), E_x
        const int hx = row ? tid + 1 : 0, hy = row ? 0 : tid - TX + 1;
        const int gx = wrapi(x0 - 1 + hx, n), gy = wrapi(y0 - 1 + hy, n);
        const int h = hy * HX + hx;
        const Al<T> phi = sm_alg<T, HS>(sP, h);
        const size_t g = (size_t)gx + (size_t)n * gy;
        if (row) {
            // E_y(x, y0-1): F(x, y0-1), F(x-1, y0-1) transported by U_x(x-1, y0-1), phi term via U_y
            const Al<T> eo = load_alg(src, ns, P_EY, g);
            const Al<T> F0 = sm_alg<T, FS>(sF, hx);
            const Al<T> t2 = transport_alg(sm_link<T, HS>(sU, 0, h - 1), sm_alg<T, FS>(sF, hx - 1));
            const Al<T> cm = icomm(phi, conj_alg(sm_link<T, HS>(sU, 1, h), sm_alg<T, HS>(sP, h + HX)));
#pragma unroll
            for (int a = 0; a < 8; a++)
                sEy[a * FT::SEY + tid] = eo.a[a] + half * dt * (tb * (F0.a[a] - t2.a[a]) - tp * cm.a[a]);
        } else {
            // E_x(x0-1, y): F(x0-1, y), F(x0-1, y-1) transported by U_y(x0-1, y-1), phi term via U_x
            const Al<T> eo = load_alg(src, ns, P_EX, g);
            const int f = hy * FX;
            const Al<T> F0 = sm_alg<T, FS>(sF, f);
            const Al<T> t1 = transport_alg(sm_link<T, HS>(sU, 1, h - HX), sm_alg<T, FS>(sF, f - FX));
            const Al<T> cm = icomm(phi, conj_alg(sm_link<T, HS>(sU, 0, h), sm_alg<T, HS>(sP, h + 1)));
#pragma unroll
            for (int a = 0; a < 8; a++)
                sEx[a * FT::SEX + (hy - 1) * (TX + 1)] = eo.a[a] + half * dt * (tb * (t1.a[a] - F0.a[a]) - tp * cm.a[a]);
        }
    }
    if (!push) return;  // uniform over the CTA
    __syncthreads();
    // phase 4: push of the tile's particles, gathering from shared memory
    const SmemSrc<T, TX, TY> S{sU, sP, sEx, sEy, sPi, x0, y0, n};
    double sx = 0.0, sy = 0.0, sz = 0.0, sc = 0.0;
    for (int k = tid; k < tcount; k += TX * TY) {
        T a0, a1, a2, a3;
        push_one_src(PA, S, perm[ts + k], a0, a1, a2, a3);
        sx += a0; sy += a1; sz += a2; sc += a3;
    }
    block_acc4(sx, sy, sz, sc, PA.acc);
}

}  // namespace glasma
