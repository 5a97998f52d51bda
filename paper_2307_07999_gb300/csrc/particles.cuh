// Colored particle-in-cell push of test particles under Wong's equations
// (Sec. 1 "Probes in Glasma", Eq. 2 of arXiv:2307.07999) and the momentum-
// broadening sums of Sec. 2 ("Quantifying the effect of Glasma").
//
// Particle state (structure of arrays, n_p entries each):
//   cell (int32, x + n*y), pid (int32, original index), ox, oy (offsets in the
//   cell, [0,1)), eta, p0x, p0y, p0z (lab momentum at formation), dpx, dpy
//   (px = p0x + dpx, py = p0y + dpy), peta (tau * p^eta), Q^a (8 planes).
// Keeping the transverse momentum as p0 + dp and the position as cell + offset
// keeps FP32 round-off relative to the change, not to the absolute value.
#pragma once
#include "field.cuh"

namespace glasma {

template <class T> struct PartSoA {
    int* cell; int* pid;
    T *ox, *oy, *eta, *p0x, *p0y, *p0z, *dpx, *dpy, *peta, *Q;  // Q: 8 planes, stride qs
    size_t qs;
};

template <class T> struct PushArgs {
    const T* fo;   // fields at step n   (U_n, phi_n, E_{n-1/2}, pi_{n-1/2})
    const T* fn;   // fields at step n+1 (E_{n+1/2}, pi_{n+1/2} used)
    int n;
    PartSoA<T> P;
    int np;
    T dtau;
    T te;          // tau_n (expanding) or 1: divides E_i and D_i phi
    T ichr;        // 1/tau_n (expanding, Christoffel term) or 0
    T teh;         // tau_{n+1/2} (expanding) or 1: eta drift
    int nsub;      // particle steps per field step (1: one step with the coefficients above)
    T hsub, tau0;  // nsub > 1: steps of hsub from tau0 = tau_n, coefficients per step
    int interp;    // gather: 0 nearest grid point, 1 cloud in cell (SUB kernels only)
    T mass;
    int expanding;
    int boris;     // momentum kick: 0 explicit (first order), 1 Boris (second order)
    T dec0, dec1;  // Boris: p_eta^ decay tau_n/tau_{n+1/2}, tau_{n+1/2}/tau_{n+1} (1 in a static box)
    double* acc;   // this step's row: {sum dpx^2, sum dpy^2, sum dpz^2, count}
    // record push (RecordSrc): the gather records the field step of this step wrote, and
    // the occupancy stamps, set to epoch_next at every particle's new cell
    const T* rec;
    int* occ;
    int epoch_next;
    // split push (ForceSrc): the Q-contracted fields of every particle, written by the force
    // kernel: 6 planes of np reals (plane stride P.qs) {Q.E_x, Q.E_y, Q.E_z, Q.B_x, Q.B_y, Q.B_z}
    T* frc;
};

template <class T> DEV M3<T> dagger(const M3<T>& A) {
    M3<T> D;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) D.m[i][j] = cj(A.m[j][i]);
    return D;
}
template <class T> DEV M3<T> mul_dn(const M3<T>& A, const M3<T>& B) {  // A^dag B
    M3<T> C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            C.m[i][j] = val(ccmac(ccmac(ccmul(A.m[0][i], B.m[0][j]), A.m[1][i], B.m[1][j]), A.m[2][i], B.m[2][j]));
    return C;
}
template <class T> DEV T dot8(const Al<T>& a, const Al<T>& b) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; k++) s = fma(a.a[k], b.a[k], s);
    return s;
}

template <class T> DEV T clamp_below_one(T v);
template <> DEV float clamp_below_one<float>(float v) { return fminf(v, 0.99999994f); }
template <> DEV double clamp_below_one<double>(double v) { return fmin(v, 0.99999999999999989); }

// Field sources of the push.  A source hands out, per particle, a view of the fields
// around the particle's cell c; the view's accessors take the offset (dx, dy) in
// {-1, 0, 1}^2 of a site from c (periodic neighbours):
//   link(d, dx, dy), links(dx, dy, ux, uy)   links at the site (U_n)
//   phi(dx, dy)                              phi at the site (phi_n)
//   eavg(d, dx, dy), piavg()                 (E_i(tau_{n-1/2}) + E_i(tau_{n+1/2})) / 2 on
//                                            the link site -> site + i, pi likewise at c
//   plaq(dx, dy) (views with kPlaq)          ImTL of the plaquette based at the site
// Global source of the unfused push: the two field buffers of step n.  PLAQ: the field
// step of step n stored the plaquettes in fo's last group (one-event paths).
template <class T, bool CG = false, bool PLAQ = false> struct GlobalSrc {
    static constexpr bool kRecord = false, kForce = false;
    const T* fo;
    const T* fn;
    int n;
    size_t ns;
    struct View {
        const T* fo;
        const T* fn;
        size_t ns;
        int n, cx, cy, xm, xp, ym, yp;
        DEV size_t at(int dx, int dy) const {
            const int x = dx < 0 ? xm : (dx > 0 ? xp : cx), y = dy < 0 ? ym : (dy > 0 ? yp : cy);
            return (size_t)x + (size_t)n * y;
        }
        DEV M3<T> link(int d, int dx, int dy) const { return load_link<T, CG>(fo, ns, d == 0 ? P_UX : P_UY, at(dx, dy)); }
        DEV void links(int dx, int dy, M3<T>& ux, M3<T>& uy) const { load_links<T, CG>(fo, ns, at(dx, dy), ux, uy); }
        DEV Al<T> phi(int dx, int dy) const { return load_alg<T, CG>(fo, ns, P_PHI, at(dx, dy)); }
        // ImTL of the plaquette based at the site, of the links of step n (written by the
        // field step of step n into the buffer it reads)
        DEV Al<T> plaq(int dx, int dy) const { return load_alg<T, CG>(fo, ns, P_F, at(dx, dy)); }
        static constexpr bool kPlaq = PLAQ;
        DEV Al<T> eavg(int d, int dx, int dy) const { return avg(d == 0 ? P_EX : P_EY, at(dx, dy)); }
        DEV Al<T> piavg() const { return avg(P_PI, at(0, 0)); }
        DEV Al<T> avg(int p, size_t s) const {
            Al<T> e = load_alg<T, CG>(fo, ns, p, s);
            const Al<T> b = load_alg<T, CG>(fn, ns, p, s);
#pragma unroll
            for (int a = 0; a < 8; a++) e.a[a] = T(0.5) * (e.a[a] + b.a[a]);
            return e;
        }
    };
    DEV View view(int cx, int cy) const {
        return View{fo, fn, ns, n, cx, cy, cx == 0 ? n - 1 : cx - 1, cx == n - 1 ? 0 : cx + 1,
                    cy == 0 ? n - 1 : cy - 1, cy == n - 1 ? 0 : cy + 1};
    }
};

// Staged source (FP32 batched push): the field groups one particle's gather reads,
// copied beforehand into a per-thread shared-memory record.  Slots (8 reals each):
//   c:      0-2 links, 3 E_x fo, 4 E_y fo, 5 E_x fn, 6 E_y fn, 7 phi, 8 pi fo, 9 pi fn
//   c-x:    10-12 links, 13 E_x fo, 14 E_x fn, 15 phi
//   c-y:    16-18 links, 19 E_y fo, 20 E_y fn, 21 phi
//   c-x-y:  22-24 links
//   c+x:    25-26 link groups 1, 2 (U_y), 27 phi
//   c+y:    28-29 link groups 0, 1 (U_x), 30 phi
//   c-x+y:  31-32 link groups 0, 1 (U_x)
//   c+x-y:  33-34 link groups 1, 2 (U_y)
// (fo: the buffer of step n, fn: of step n+1; groups as in the field buffer layout.)
constexpr int STAGE_SLOTS = 35;
// slot of field group g (0..6) of buffer b (0: fo, 1: fn) at offset (dx, dy); -1 if not staged
__host__ __device__ constexpr int stage_slot(int dx, int dy, int g, int b) {
    if (g <= 2) {  // links (fo only)
        if (dx == 0 && dy == 0) return g;
        if (dx == -1 && dy == 0) return 10 + g;
        if (dx == 0 && dy == -1) return 16 + g;
        if (dx == -1 && dy == -1) return 22 + g;
        if (dx == 1 && dy == 0) return g >= 1 ? 24 + g : -1;
        if (dx == 0 && dy == 1) return g <= 1 ? 28 + g : -1;
        if (dx == -1 && dy == 1) return g <= 1 ? 31 + g : -1;
        if (dx == 1 && dy == -1) return g >= 1 ? 32 + g : -1;
        return -1;
    }
    if (g == 5) {  // phi (fo)
        if (dx == 0 && dy == 0) return 7;
        if (dx == -1 && dy == 0) return 15;
        if (dx == 0 && dy == -1) return 21;
        if (dx == 1 && dy == 0) return 27;
        if (dx == 0 && dy == 1) return 30;
        return -1;
    }
    if (g == 6) return (dx == 0 && dy == 0) ? 8 + b : -1;  // pi
    // E_x (g = 3), E_y (g = 4)
    if (dx == 0 && dy == 0) return 3 + (g - 3) + 2 * b;
    if (dx == -1 && dy == 0 && g == 3) return 13 + b;
    if (dx == 0 && dy == -1 && g == 4) return 19 + b;
    return -1;
}
template <class T> struct StagedSrc {
    static constexpr bool kRecord = false, kForce = false;
    static constexpr int STRIDE = STAGE_SLOTS * 8 + (sizeof(T) == 4 ? 4 : 2);  // bank-spread record stride
    const T* rec;  // this thread's record
    struct View {
        const T* r;
        DEV const T* grp(int dx, int dy, int g, int b = 0) const { return r + 8 * stage_slot(dx, dy, g, b); }
        DEV M3<T> link(int d, int dx, int dy) const {
            M3<T> U;
            if (d == 0) {
                const T* a = grp(dx, dy, 0);
                const T* b = grp(dx, dy, 1);
#pragma unroll
                for (int e = 0; e < 4; e++) put_entry(U, e, a[2 * e], a[2 * e + 1]);
                put_entry(U, 4, b[0], b[1]);
                put_entry(U, 5, b[2], b[3]);
            } else {
                const T* a = grp(dx, dy, 1);
                const T* b = grp(dx, dy, 2);
                put_entry(U, 0, a[4], a[5]);
                put_entry(U, 1, a[6], a[7]);
#pragma unroll
                for (int e = 0; e < 4; e++) put_entry(U, 2 + e, b[2 * e], b[2 * e + 1]);
            }
            complete_row2(U);
            return U;
        }
        DEV void links(int dx, int dy, M3<T>& ux, M3<T>& uy) const {
            ux = link(0, dx, dy);
            uy = link(1, dx, dy);
        }
        DEV Al<T> phi(int dx, int dy) const { return ld(grp(dx, dy, 5)); }
        static constexpr bool kPlaq = false;  // no plaquettes staged: the clover is formed here
        DEV Al<T> eavg(int d, int dx, int dy) const { return avg(grp(dx, dy, 3 + d, 0), grp(dx, dy, 3 + d, 1)); }
        DEV Al<T> piavg() const { return avg(grp(0, 0, 6, 0), grp(0, 0, 6, 1)); }
        DEV static Al<T> ld(const T* p) {
            Al<T> x;
#pragma unroll
            for (int a = 0; a < 8; a++) x.a[a] = p[a];
            return x;
        }
        DEV static Al<T> avg(const T* p, const T* q) {
            Al<T> x;
#pragma unroll
            for (int a = 0; a < 8; a++) x.a[a] = T(0.5) * (p[a] + q[a]);
            return x;
        }
    };
    DEV View view(int, int) const { return View{rec}; }
};

// Plaquette k (0..3) of the clover at the view's cell, counter-clockwise from the cell,
// written as (L0 L1)(L3 L2)^dag:
//   0 +x,+y: U_x(c) U_y(c+x) [U_y(c) U_x(c+y)]^dag
//   1 +y,-x: U_y(c) U_x(c-x+y)^dag U_y(c-x)^dag U_x(c-x) = [U_y(c) U_x(c-x+y)^dag] [U_x(c-x)^dag U_y(c-x)]^dag
//   2 -x,-y: U_x(c-x)^dag U_y(c-x-y)^dag U_x(c-x-y) U_y(c-y) = [U_x(c-x)^dag U_y(c-x-y)^dag] [U_y(c-y)^dag U_x(c-x-y)^dag]^dag
//   3 -y,+x: U_y(c-y)^dag U_x(c-y) U_y(c+x-y) U_x(c)^dag = [U_y(c-y)^dag U_x(c-y)] [U_x(c) U_y(c+x-y)^dag]^dag
template <class T, class V> DEV M3<T> clover_plaquette(const V& C, int k) {
    M3<T> A, B;
    switch (k) {
        case 0: A = mul(C.link(0, 0, 0), C.link(1, 1, 0)); B = mul(C.link(1, 0, 0), C.link(0, 0, 1)); break;
        case 1: A = mul_nd(C.link(1, 0, 0), C.link(0, -1, 1)); B = mul_dn(C.link(0, -1, 0), C.link(1, -1, 0)); break;
        case 2: A = mul_dn(C.link(0, -1, 0), dagger(C.link(1, -1, -1))); B = mul_dn(C.link(1, 0, -1), dagger(C.link(0, -1, -1))); break;
        default: A = mul_dn(C.link(1, 0, -1), C.link(0, 0, -1)); B = mul_nd(C.link(0, 0, 0), C.link(1, 1, -1)); break;
    }
    return mul_nd(A, B);
}

// Q-contracted site-centred fields at the particle's cell for the push of step n:
// qE = Q.(E_x, E_y, E_z), qB = Q.(B_x, B_y, B_z)
//
// Views with the stored plaquettes (kPlaq): the fields at c-x and c-y reach c by a
// transport U^dag X U with the link from there to c, and Q.(U^dag X U) = (U Q U^dag).X,
// so Q is carried to c-x and c-y once and contracted there with E, phi and the plaquette.
// The clover leaves other than the plaquette at c are the plaquettes at c-x, c-y and
// c-x-y carried to c (cyclic rotations of those loops): by U_x(c-x), by U_y(c-y), and by
// V = U_x(c-x-y) U_y(c-y) (ImTL commutes with the conjugation), so Q at c-y is carried on
// by U_x(c-x-y).  Five transports of Q replace six of fields and the twelve products of
// the four leaves; the gather reads six sites instead of eight.
template <class T, class V>
DEV void gather_qf_view(const V& C, T te, const Al<T>& q, T qE[3], T qB[3]) {
    const T half = T(0.5);
    if constexpr (V::kPlaq) {
        T bz;
        {
            const Al<T> ql = conj_alg(C.link(0, -1, 0), q);  // Q carried to c-x
            qE[0] = half * (dot8(q, C.eavg(0, 0, 0)) + dot8(ql, C.eavg(0, -1, 0))) / te;
            qB[1] = -half * dot8(ql, C.phi(-1, 0));
            bz = dot8(q, C.plaq(0, 0)) + dot8(ql, C.plaq(-1, 0));
        }
        {
            const Al<T> qb = conj_alg(C.link(1, 0, -1), q);  // Q carried to c-y
            qE[1] = half * (dot8(q, C.eavg(1, 0, 0)) + dot8(qb, C.eavg(1, 0, -1))) / te;
            qB[0] = half * dot8(qb, C.phi(0, -1));
            bz += dot8(qb, C.plaq(0, -1));
            bz += dot8(conj_alg(C.link(0, -1, -1), qb), C.plaq(-1, -1));  // on to c-x-y
        }
        qE[2] = dot8(q, C.piavg());
        // B_y = +D_x phi / tau,  B_x = -D_y phi / tau (central differences); phi at c+x and
        // c+y reaches c by U phi U^dag: Q.(U phi U^dag) = (U^dag Q U).phi
        qB[1] = (qB[1] + half * dot8(transport_alg(C.link(0, 0, 0), q), C.phi(1, 0))) / te;
        qB[0] = (qB[0] - half * dot8(transport_alg(C.link(1, 0, 0), q), C.phi(0, 1))) / te;
        qB[2] = -T(0.25) * bz;
        return;
    }
    // Every field is read from the view where it is used and contracted with Q at once
    // (Q.X is linear in X), so that few 3x3 matrices are live at a time.
    // electric: the two links touching c, time-centred, transported to c
    qE[0] = half * (dot8(q, C.eavg(0, 0, 0)) + dot8(q, transport_alg(C.link(0, -1, 0), C.eavg(0, -1, 0)))) / te;
    qE[1] = half * (dot8(q, C.eavg(1, 0, 0)) + dot8(q, transport_alg(C.link(1, 0, -1), C.eavg(1, 0, -1)))) / te;
    qE[2] = dot8(q, C.piavg());
    // magnetic from phi: covariant central differences
    // B_y = +D_x phi / tau,  B_x = -D_y phi / tau
    qB[1] = half * (dot8(q, conj_alg(C.link(0, 0, 0), C.phi(1, 0))) -
                    dot8(q, transport_alg(C.link(0, -1, 0), C.phi(-1, 0)))) / te;
    qB[0] = -half * (dot8(q, conj_alg(C.link(1, 0, 0), C.phi(0, 1))) -
                     dot8(q, transport_alg(C.link(1, 0, -1), C.phi(0, -1)))) / te;
    // B_z = -F_xy, F_xy = clover average of the four plaquettes based at c (one per
    // iteration, not unrolled: one copy of the products, fewer live matrices)
    T bz = T(0);
#pragma unroll 1
    for (int k = 0; k < 4; k++) bz += dot8(q, im_tl(clover_plaquette<T>(C, k)));
    qB[2] = -T(0.25) * bz;
}

// Record source (batched push after a field step that wrote gather records, see the
// record layout in field.cuh): the site-centred fields of the particle's cell come from
// its record, one contiguous read, instead of 35 scattered field groups.  The pieces are
// those gather_qf_view forms, contracted with Q in the same order; the pieces of the
// neighbours c-x and c-y were stored untransported with their links, so Q is carried
// there instead: Q.(U^dag X U) = (U Q U^dag).X.  Links for cell crossings and phi at
// the cell come from the field buffer and the record.
template <class T> struct RecordSrc {
    static constexpr bool kRecord = true, kForce = false;
    const T* rec;
    GlobalSrc<T> g;
    struct View {
        const T* r;  // this cell's record
        typename GlobalSrc<T>::View gv;
        DEV Al<T> grp(int slot) const {
            const V8<T> v = ld8<false>(r + 8 * slot);
            Al<T> x;
#pragma unroll
            for (int a = 0; a < 8; a++) x.a[a] = v.v[a];
            return x;
        }
        DEV M3<T> rlink(int slot) const {
            const V8<T> a = ld8<false>(r + 8 * slot);
            const V4<T> b = ld4<false>(r + 8 * (slot + 1));
            M3<T> U;
#pragma unroll
            for (int e = 0; e < 4; e++) put_entry(U, e, a.v[2 * e], a.v[2 * e + 1]);
            put_entry(U, 4, b.v[0], b.v[1]);
            put_entry(U, 5, b.v[2], b.v[3]);
            complete_row2(U);
            return U;
        }
        DEV M3<T> link(int d, int dx, int dy) const { return gv.link(d, dx, dy); }
        DEV Al<T> phi(int, int) const { return grp(R_PHI); }  // used at the cell itself only
        DEV void gather(T te, const Al<T>& q, T qE[3], T qB[3]) const {
            const T half = T(0.5);
            const Al<T> ql = conj_alg(rlink(R_UXL), q);  // Q carried to c-x
            const Al<T> qb = conj_alg(rlink(R_UYB), q);  // Q carried to c-y
            qE[0] = half * (dot8(q, grp(R_EX)) + dot8(ql, grp(R_EXL))) / te;
            qE[1] = half * (dot8(q, grp(R_EY)) + dot8(qb, grp(R_EYB))) / te;
            qE[2] = dot8(q, grp(R_PI));
            qB[1] = half * (dot8(q, grp(R_PSX)) - dot8(q, grp(R_CHX))) / te;
            qB[0] = -half * (dot8(q, grp(R_PSY)) - dot8(q, grp(R_CHY))) / te;
            // clover leaves in the order of clover_plaquette: +x+y, +y-x, -x-y, -y+x
            T bz = dot8(q, grp(R_F0));
            bz += dot8(q, grp(R_T2));
            bz += dot8(ql, grp(R_T1L));
            bz += dot8(q, grp(R_T1));
            qB[2] = -T(0.25) * bz;
        }
    };
    DEV View view(int cx, int cy) const {
        return View{rec + ((size_t)cx + (size_t)g.n * cy) * REC_STRIDE * 8, g.view(cx, cy)};
    }
};

// Force source (second kernel of the split push): the Q-contracted fields of the particle,
// gathered by the force kernel and stored per particle (PushArgs::frc); phi at the cell and
// the links of cell crossings come from the field buffer as in the unfused push.
template <class T> struct ForceSrc : GlobalSrc<T> {
    static constexpr bool kRecord = false, kForce = true;
};

// Cloud-in-cell gather: the Q-contracted fields of the four sites around the particle
// (c, c+x, c+y, c+x+y) carried to c, with bilinear weights in the offsets (ox, oy).
// Carrying the field F(s) to c is W F(s) W^dag with W the links from c to s (x before y
// for the diagonal site); Q.(W F W^dag) = (W^dag Q W).F, so Q is carried to each site
// instead (three transports of one 8-vector rather than eighteen).  The source must
// serve views at any cell (GlobalSrc).
template <class T, class S>
DEV void gather_qf_cic(const S& F, int n, int cx, int cy, T ox, T oy, T te, const Al<T>& q, T qE[3], T qB[3]) {
    const int xp = cx == n - 1 ? 0 : cx + 1, yp = cy == n - 1 ? 0 : cy + 1;
#pragma unroll
    for (int i = 0; i < 3; i++) { qE[i] = T(0); qB[i] = T(0); }
    // one site per iteration, not unrolled: one copy of the gather (four inlined copies spill)
#pragma unroll 1
    for (int k = 0; k < 4; k++) {
        const auto C = F.view(cx, cy);
        Al<T> qk = q;
        if (k & 1) qk = transport_alg(C.link(0, 0, 0), qk);                   // c -> c+x
        if (k & 2) qk = transport_alg(C.link(1, (k & 1) ? 1 : 0, 0), qk);     // -> +y (x first)
        const T w = ((k & 1) ? ox : T(1) - ox) * ((k & 2) ? oy : T(1) - oy);
        T e[3], b[3];
        gather_qf_view(F.view((k & 1) ? xp : cx, (k & 2) ? yp : cy), te, qk, e, b);
#pragma unroll
        for (int i = 0; i < 3; i++) { qE[i] = fma(w, e[i], qE[i]); qB[i] = fma(w, b[i], qB[i]); }
    }
}

// The site-centred fields at the view's cell, as 8-vectors (the same formulas as
// gather_qf_view, which contracts each with Q as soon as it is read):
// E = (E_x, E_y, E_z), B = (B_x, B_y, B_z)
template <class T, class V> DEV void site_E(const V& C, T te, Al<T> E[3]) {
    const T half = T(0.5);
    {
        const Al<T> a = C.eavg(0, 0, 0), b = transport_alg(C.link(0, -1, 0), C.eavg(0, -1, 0));
#pragma unroll
        for (int k = 0; k < 8; k++) E[0].a[k] = half * (a.a[k] + b.a[k]) / te;
    }
    {
        const Al<T> a = C.eavg(1, 0, 0), b = transport_alg(C.link(1, 0, -1), C.eavg(1, 0, -1));
#pragma unroll
        for (int k = 0; k < 8; k++) E[1].a[k] = half * (a.a[k] + b.a[k]) / te;
    }
    E[2] = C.piavg();
}
template <class T, class V> DEV void site_fields(const V& C, T te, Al<T> E[3], Al<T> B[3]) {
    const T half = T(0.5);
    site_E(C, te, E);
    {
        const Al<T> fw = conj_alg(C.link(0, 0, 0), C.phi(1, 0)), bw = transport_alg(C.link(0, -1, 0), C.phi(-1, 0));
#pragma unroll
        for (int k = 0; k < 8; k++) B[1].a[k] = half * (fw.a[k] - bw.a[k]) / te;  // +D_x phi / tau
    }
    {
        const Al<T> fw = conj_alg(C.link(1, 0, 0), C.phi(0, 1)), bw = transport_alg(C.link(1, 0, -1), C.phi(0, -1));
#pragma unroll
        for (int k = 0; k < 8; k++) B[0].a[k] = -half * (fw.a[k] - bw.a[k]) / te;  // -D_y phi / tau
    }
    Al<T> acc;
    if constexpr (V::kPlaq) {
        // the stored plaquettes at c, c-x, c-y, c-x-y, the last three carried to c (the clover
        // leaves, as in gather_qf_view): U^dag F U with U_x(c-x), U_y(c-y), and U_x(c-x-y)
        // then U_y(c-y)
        acc = C.plaq(0, 0);
        const Al<T> t1 = transport_alg(C.link(0, -1, 0), C.plaq(-1, 0));
        const Al<T> t3 = transport_alg(C.link(1, 0, -1), C.plaq(0, -1));
#pragma unroll
        for (int a = 0; a < 8; a++) acc.a[a] += t1.a[a] + t3.a[a];
        const Al<T> t2 = transport_alg(C.link(1, 0, -1), transport_alg(C.link(0, -1, -1), C.plaq(-1, -1)));
#pragma unroll
        for (int a = 0; a < 8; a++) acc.a[a] += t2.a[a];
    } else {
#pragma unroll
        for (int a = 0; a < 8; a++) acc.a[a] = T(0);
#pragma unroll 1
        for (int k = 0; k < 4; k++) {
            const Al<T> t = im_tl(clover_plaquette<T>(C, k));
#pragma unroll
            for (int a = 0; a < 8; a++) acc.a[a] += t.a[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 8; a++) B[2].a[a] = -T(0.25) * acc.a[a];
}

// one particle: gather, kick, drift, color transport; returns its broadening terms.
// SUB: the step is taken as A.nsub particle steps of A.hsub, each gathering the step's
// fields at the particle's current cell, by nearest grid point or cloud in cell
// (A.interp); the source must serve any cell (GlobalSrc).
// Without SUB the loop runs once with the host's coefficients (the kernels of the
// default path are compiled without it: the loop's carried state costs registers).
template <class T, class S, bool CG = false, bool SUB = false>
DEV void push_one_src(const PushArgs<T>& A, const S& F, int j, T& sx, T& sy, T& sz, T& sc) {
    const PartSoA<T>& P = A.P;
    const int n = A.n;
    const int cell = CG ? __ldcg(P.cell + j) : P.cell[j];
    int cx = cell % n, cy = cell / n;
    Al<T> q;
#pragma unroll
    for (int a = 0; a < 8; a++) q.a[a] = CG ? __ldcg(P.Q + (size_t)a * P.qs + j) : P.Q[(size_t)a * P.qs + j];
    const T p0x = P.p0x[j], p0y = P.p0y[j];  // constant during a run
    T dpx = CG ? __ldcg(P.dpx + j) : P.dpx[j], dpy = CG ? __ldcg(P.dpy + j) : P.dpy[j];
    T pz = CG ? __ldcg(P.peta + j) : P.peta[j];
    T ox, oy, eta;
    if (SUB) {  // the cloud-in-cell gather needs the offsets first
        ox = CG ? __ldcg(P.ox + j) : P.ox[j];
        oy = CG ? __ldcg(P.oy + j) : P.oy[j];
        eta = CG ? __ldcg(P.eta + j) : P.eta[j];
    }
    const T m2 = A.mass * A.mass;
    T px, py, ptn;
    const int nsub = SUB ? A.nsub : 1;
    for (int k = 0; k < nsub; k++) {
        T h = A.dtau, ichr = A.ichr, teh = A.teh, dec0 = A.dec0, dec1 = A.dec1;
        if (SUB && nsub > 1) {
            h = A.hsub;
            if (A.expanding) {
                const T tk = A.tau0 + T(k) * h, tm = tk + T(0.5) * h;
                ichr = T(1) / tk;
                teh = tm;
                dec0 = tk / tm;
                dec1 = tm / (tk + h);
            }
        }
        T qE[3], qB[3];
        const auto C = F.view(cx, cy);
        if constexpr (S::kForce) {
#pragma unroll
            for (int i = 0; i < 3; i++) {
                qE[i] = A.frc[(size_t)i * P.qs + j];
                qB[i] = A.frc[(size_t)(3 + i) * P.qs + j];
            }
        } else if constexpr (S::kRecord)
            C.gather(A.te, q, qE, qB);
        else if (SUB && A.interp)
            gather_qf_cic(F, n, cx, cy, ox, oy, A.te, q, qE, qB);
        else
            gather_qf_view(C, A.te, q, qE, qB);
        px = p0x + dpx;
        py = p0y + dpy;
        if (!A.boris) {
            // explicit: p += h [Q.E + (p / p^tau) x Q.B] - h p_eta^ / tau e_eta
            const T pt = sqrt(m2 + px * px + py * py + pz * pz);
            const T ipt = pt > T(0) ? T(1) / pt : T(0);
            const T fx = qE[0] + (py * qB[2] - pz * qB[1]) * ipt;
            const T fy = qE[1] + (pz * qB[0] - px * qB[2]) * ipt;
            const T fz = qE[2] + (px * qB[1] - py * qB[0]) * ipt - pz * ichr;
            dpx += h * fx;
            dpy += h * fy;
            pz += h * fz;
        } else {
            // Boris (1970): the Christoffel decay of p_eta^ over the first half step (exact for
            // a free particle), half electric kick, rotation about Q.B by the angle of
            // t = (h/2) Q.B / p^tau (|p| unchanged), half electric kick, decay over the second
            // half step.  The transverse change is accumulated into dp, so FP32 round-off
            // stays relative to the change.
            const T hh = T(0.5) * h;
            pz *= dec0;
            const T mx = px + hh * qE[0], my = py + hh * qE[1], mz = pz + hh * qE[2];
            const T g = sqrt(m2 + mx * mx + my * my + mz * mz);
            const T ig = g > T(0) ? hh / g : T(0);
            const T tx = qB[0] * ig, ty = qB[1] * ig, tz = qB[2] * ig;
            const T ux = mx + (my * tz - mz * ty), uy = my + (mz * tx - mx * tz), uz = mz + (mx * ty - my * tx);
            const T sf = T(2) / (T(1) + tx * tx + ty * ty + tz * tz);
            dpx += h * qE[0] + sf * (uy * tz - uz * ty);
            dpy += h * qE[1] + sf * (uz * tx - ux * tz);
            pz = (mz + sf * (ux * ty - uy * tx) + hh * qE[2]) * dec1;
        }
        px = p0x + dpx;
        py = p0y + dpy;
        ptn = sqrt(m2 + px * px + py * py + pz * pz);
        const T iptn = ptn > T(0) ? T(1) / ptn : T(0);
        if (!SUB && k == 0) {  // loaded here, after the gather, to keep them out of its live range
            ox = CG ? __ldcg(P.ox + j) : P.ox[j];
            oy = CG ? __ldcg(P.oy + j) : P.oy[j];
            eta = CG ? __ldcg(P.eta + j) : P.eta[j];
        }
        ox += h * px * iptn;
        oy += h * py * iptn;
        const T deta = h * pz * iptn / teh;
        // color: rotation along eta at the old cell, then across the x face, then the y face
        {
            Al<T> e;
            const Al<T> ph = C.phi(0, 0);
#pragma unroll
            for (int a = 0; a < 8; a++) e.a[a] = -deta * ph.a[a];
            q = alg(conj_by(expi(herm(e)), herm(q)));
        }
        int nx = cx, ny = cy, ddx = 0;
        if (ox >= T(1)) {
            q = transport_alg(C.link(0, 0, 0), q);
            ox -= T(1);
            nx = cx == n - 1 ? 0 : cx + 1;
            ddx = 1;
        } else if (ox < T(0)) {
            nx = cx == 0 ? n - 1 : cx - 1;
            ddx = -1;
            q = conj_alg(C.link(0, -1, 0), q);
            ox = clamp_below_one(ox + T(1));
        }
        if (oy >= T(1)) {
            q = transport_alg(C.link(1, ddx, 0), q);
            oy -= T(1);
            ny = cy == n - 1 ? 0 : cy + 1;
        } else if (oy < T(0)) {
            ny = cy == 0 ? n - 1 : cy - 1;
            q = conj_alg(C.link(1, ddx, -1), q);
            oy = clamp_below_one(oy + T(1));
        }
        cx = nx;
        cy = ny;
        eta += deta;
    }
    P.cell[j] = cx + n * cy;
    if constexpr (S::kRecord) A.occ[cx + n * cy] = A.epoch_next;  // the next field step writes its record
    P.ox[j] = ox;
    P.oy[j] = oy;
    P.eta[j] = eta;
    P.dpx[j] = dpx;
    P.dpy[j] = dpy;
    P.peta[j] = pz;
#pragma unroll
    for (int a = 0; a < 8; a++) P.Q[(size_t)a * P.qs + j] = q.a[a];
    // broadening terms: dp_i^2 = p_i^2 - p_i(tau_form)^2, lab p_z.  The transverse terms
    // are factored, dp (2 p0 + dp), so they carry no cancellation and are computed in the
    // working precision; so is the longitudinal one when p_z(tau_form) = 0 (every particle
    // formed at eta = 0 with p_eta^ = 0).  Otherwise p_z^2 - p0z^2 can cancel and is
    // taken in FP64.  The sums over particles are FP64 (block_acc4).
    const T p0z = P.p0z[j];
    if (p0z == T(0)) {
        const T pzl = A.expanding ? ptn * sinh(eta) + pz * cosh(eta) : pz;
        sz = pzl * pzl;
    } else {
        const double pzl = A.expanding ? (double)ptn * sinh((double)eta) + (double)pz * cosh((double)eta)
                                       : (double)pz;
        sz = (T)(pzl * pzl - (double)p0z * (double)p0z);
    }
    sx = dpx * fma(T(2), p0x, dpx);
    sy = dpy * fma(T(2), p0y, dpy);
    sc = T(1);
}

template <class T, bool CG = false, bool SUB = false, bool PLAQ = false>
DEV void push_one(const PushArgs<T>& A, int j, T& sx, T& sy, T& sz, T& sc) {
    GlobalSrc<T, CG, PLAQ> F{A.fo, A.fn, A.n, (size_t)A.n * A.n};
    push_one_src<T, GlobalSrc<T, CG, PLAQ>, CG, SUB>(A, F, j, sx, sy, sz, sc);
}

// warp -> block -> one FP64 atomic per block and term (any block shape, at most 256
// threads, a multiple of 32).  FP64 terms: FP64 shuffles and sums.
DEV void block_acc4(double sx, double sy, double sz, double sc, double* acc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        sz += __shfl_down_sync(0xffffffffu, sz, o);
        sc += __shfl_down_sync(0xffffffffu, sc, o);
    }
    __shared__ double red[4][8];
    const int lt = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    const int w = lt >> 5, l = lt & 31;
    if (l == 0) { red[0][w] = sx; red[1][w] = sy; red[2][w] = sz; red[3][w] = sc; }
    __syncthreads();
    if (lt < 4) {
        double t = 0.0;
        for (int k = 0; k < nw; k++) t += red[lt][k];
        atomicAdd(acc + lt, t);
    }
}

// FP32 terms: the warp sums are compensated (Knuth's TwoSum keeps the rounding error of
// every addition in a second FP32 word), so each warp's sum is the exact sum of its 32
// terms to about 2^-48 relative, formed without FP64 arithmetic (slow on GB300); the
// warp sums then go to FP64 and on as above.  The count term is an exact small integer.
DEV void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
DEV void block_acc4(float tx, float ty, float tz, float tc, double* acc) {
    float h[3] = {tx, ty, tz}, l[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float oh = __shfl_down_sync(0xffffffffu, h[k], o), ol = __shfl_down_sync(0xffffffffu, l[k], o);
            float sum, err;
            two_sum(h[k], oh, sum, err);
            h[k] = sum;
            l[k] += ol + err;
        }
        tc += __shfl_down_sync(0xffffffffu, tc, o);
    }
    __shared__ double red[4][8];
    const int lt = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    const int w = lt >> 5, ln = lt & 31;
    if (ln == 0) {
#pragma unroll
        for (int k = 0; k < 3; k++) red[k][w] = (double)h[k] + (double)l[k];
        red[3][w] = (double)tc;
    }
    __syncthreads();
    if (lt < 4) {
        double t = 0.0;
        for (int k = 0; k < nw; k++) t += red[lt][k];
        atomicAdd(acc + lt, t);
    }
}

// one event's push, NT threads per block and at least MINB blocks per SM (see launch_push)
template <class T, bool SUB, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_push(PushArgs<T> A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    T sx = T(0), sy = T(0), sz = T(0), sc = T(0);
    if (j < A.np) push_one<T, false, SUB, true>(A, j, sx, sy, sz, sc);
    block_acc4(sx, sy, sz, sc, A.acc);
}

// Several ensembles of one event in one launch: block b pushes the particles
// [(b / n) NT, (b / n + 1) NT) of ensemble b % n, so the ensembles' blocks interleave.
// Each ensemble sorted by cell, blocks at the same position gather from neighbouring
// cells, and the field lines they read come from DRAM once for all the ensembles.
constexpr int PUSH_PACK = 8;
template <class T> struct PushPack {
    PushArgs<T> a[PUSH_PACK];
    int n;
};
template <class T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_push_pack(const __grid_constant__ PushPack<T> P) {
    const int e = (int)(blockIdx.x % (unsigned)P.n), j0 = (int)(blockIdx.x / (unsigned)P.n) * NT;
    const PushArgs<T>& A = P.a[e];
    if (j0 >= A.np) return;  // uniform over the block: this ensemble has fewer particles
    const int j = j0 + (int)threadIdx.x;
    T sx = T(0), sy = T(0), sz = T(0), sc = T(0);
    if (j < A.np) push_one<T, false, false, true>(A, j, sx, sy, sz, sc);
    block_acc4(sx, sy, sz, sc, A.acc);
}

// batched over events: one item per 256 particles of an event, pushed by 256 / NT blocks
// of NT threads; args[ev] of this step (acc == nullptr marks an event whose particles
// are not pushed at this step)
struct PushItem { int ev, j0; };
template <class T, int NT, int MINB, bool MULTI = false>
__global__ void __launch_bounds__(NT, MINB) k_push_batched(const PushArgs<T>* __restrict__ args,
                                                           const PushItem* __restrict__ items) {
    static_assert(256 % NT == 0 && NT % 32 == 0, "push block");
    constexpr int SUB = 256 / NT;
    const PushItem it = items[blockIdx.x / SUB];
    const PushArgs<T>& A = args[it.ev];  // read where used: a copy held ~50 registers
    if (A.acc == nullptr) return;
    const int j = it.j0 + (int)(blockIdx.x % SUB) * NT + threadIdx.x;
    T sx = T(0), sy = T(0), sz = T(0), sc = T(0);
    if (j < A.np) push_one<T, false, MULTI>(A, j, sx, sy, sz, sc);
    block_acc4(sx, sy, sz, sc, A.acc);
}

// batched record push: as k_push_batched, the fields from the gather records
template <class T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_push_record(const PushArgs<T>* __restrict__ args,
                                                          const PushItem* __restrict__ items) {
    static_assert(256 % NT == 0 && NT % 32 == 0, "push block");
    constexpr int SUB = 256 / NT;
    const PushItem it = items[blockIdx.x / SUB];
    const PushArgs<T>& A = args[it.ev];  // read where used: a copy held ~50 registers
    if (A.acc == nullptr) return;
    const int j = it.j0 + (int)(blockIdx.x % SUB) * NT + threadIdx.x;
    T sx = T(0), sy = T(0), sz = T(0), sc = T(0);
    if (j < A.np) {
        const RecordSrc<T> F{A.rec, GlobalSrc<T>{A.fo, A.fn, A.n, (size_t)A.n * A.n}};
        push_one_src<T, RecordSrc<T>>(A, F, j, sx, sy, sz, sc);
    }
    block_acc4(sx, sy, sz, sc, A.acc);
}

// Split push: the force kernel gathers the fields of each particle's cell and stores their
// Q-contractions (6 reals per particle); the move kernel then kicks, drifts and rotates the
// particle from them.  The gather, the part that waits on scattered loads, runs in a kernel
// with fewer registers and so more resident warps than the whole push.
template <class T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_push_force(const PushArgs<T>* __restrict__ args,
                                                         const PushItem* __restrict__ items) {
    static_assert(256 % NT == 0 && NT % 32 == 0, "push block");
    constexpr int SUB = 256 / NT;
    const PushItem it = items[blockIdx.x / SUB];
    const PushArgs<T>& A = args[it.ev];
    if (A.acc == nullptr) return;
    const int j = it.j0 + (int)(blockIdx.x % SUB) * NT + threadIdx.x;
    if (j >= A.np) return;
    const PartSoA<T>& P = A.P;
    const int n = A.n;
    const int cell = P.cell[j];
    Al<T> q;
#pragma unroll
    for (int a = 0; a < 8; a++) q.a[a] = P.Q[(size_t)a * P.qs + j];
    const GlobalSrc<T> F{A.fo, A.fn, n, (size_t)n * n};
    T qE[3], qB[3];
    gather_qf_view(F.view(cell % n, cell / n), A.te, q, qE, qB);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        A.frc[(size_t)i * P.qs + j] = qE[i];
        A.frc[(size_t)(3 + i) * P.qs + j] = qB[i];
    }
}
template <class T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_push_move(const PushArgs<T>* __restrict__ args,
                                                        const PushItem* __restrict__ items) {
    static_assert(256 % NT == 0 && NT % 32 == 0, "push block");
    constexpr int SUB = 256 / NT;
    const PushItem it = items[blockIdx.x / SUB];
    const PushArgs<T>& A = args[it.ev];  // read where used: a copy held ~50 registers
    if (A.acc == nullptr) return;
    const int j = it.j0 + (int)(blockIdx.x % SUB) * NT + threadIdx.x;
    T sx = T(0), sy = T(0), sz = T(0), sc = T(0);
    if (j < A.np) {
        const ForceSrc<T> F{{A.fo, A.fn, A.n, (size_t)A.n * A.n}};
        push_one_src<T, ForceSrc<T>>(A, F, j, sx, sy, sz, sc);
    }
    block_acc4(sx, sy, sz, sc, A.acc);
}

// ---------------------------------------------------------------- staged batched push
// Each thread first copies the 35 field groups of its particle's gather (StagedSrc) into
// its shared-memory record with cp.async, all copies in flight at once, then pushes
// from shared memory: the scattered loads overlap instead of waiting in turn.
struct StageEntry { int dx, dy, g, b; };
// the field group in slot k: offset (dx, dy) of its site, group g, buffer b
__host__ __device__ constexpr StageEntry stage_entry(int k) {
    constexpr int E[STAGE_SLOTS][4] = {
        {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 2, 0}, {0, 0, 3, 0}, {0, 0, 4, 0}, {0, 0, 3, 1}, {0, 0, 4, 1},
        {0, 0, 5, 0}, {0, 0, 6, 0}, {0, 0, 6, 1},
        {-1, 0, 0, 0}, {-1, 0, 1, 0}, {-1, 0, 2, 0}, {-1, 0, 3, 0}, {-1, 0, 3, 1}, {-1, 0, 5, 0},
        {0, -1, 0, 0}, {0, -1, 1, 0}, {0, -1, 2, 0}, {0, -1, 4, 0}, {0, -1, 4, 1}, {0, -1, 5, 0},
        {-1, -1, 0, 0}, {-1, -1, 1, 0}, {-1, -1, 2, 0},
        {1, 0, 1, 0}, {1, 0, 2, 0}, {1, 0, 5, 0},
        {0, 1, 0, 0}, {0, 1, 1, 0}, {0, 1, 5, 0},
        {-1, 1, 0, 0}, {-1, 1, 1, 0},
        {1, -1, 1, 0}, {1, -1, 2, 0}};
    return StageEntry{E[k][0], E[k][1], E[k][2], E[k][3]};
}
constexpr bool stage_table_consistent() {
    for (int k = 0; k < STAGE_SLOTS; k++) {
        const StageEntry e = stage_entry(k);
        if (stage_slot(e.dx, e.dy, e.g, e.b) != k) return false;
    }
    return true;
}
static_assert(stage_table_consistent(), "staged gather: slot table and lookup disagree");

DEV void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
DEV void cp_async_wait_all() { asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory"); }

constexpr int PUSH_PPB = 32;  // particles (threads) per block of the staged push; 6 blocks per SM
static_assert(256 % PUSH_PPB == 0 && PUSH_PPB % 32 == 0, "staged push block");
template <class T> constexpr size_t push_staged_smem() { return (size_t)PUSH_PPB * StagedSrc<T>::STRIDE * sizeof(T); }

template <class T>
__global__ void __launch_bounds__(PUSH_PPB, 6)
k_push_staged(const PushArgs<T>* __restrict__ args, const PushItem* __restrict__ items) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int SUB = 256 / PUSH_PPB;
    const PushItem it = items[blockIdx.x / SUB];
    const PushArgs<T>& A = args[it.ev];  // read where used: a copy held ~50 registers
    if (A.acc == nullptr) return;  // uniform over the block
    const int j = it.j0 + (int)(blockIdx.x % SUB) * PUSH_PPB + threadIdx.x;
    T* rec = reinterpret_cast<T*>(smem) + (size_t)threadIdx.x * StagedSrc<T>::STRIDE;
    T sx = T(0), sy = T(0), sz = T(0), sc = T(0);
    if (j < A.np) {
        const int n = A.n;
        const size_t ns = (size_t)n * n;
        const int cell = A.P.cell[j];
        const int cx = cell % n, cy = cell / n;
        const int xm = cx == 0 ? n - 1 : cx - 1, xp = cx == n - 1 ? 0 : cx + 1;
        const int ym = cy == 0 ? n - 1 : cy - 1, yp = cy == n - 1 ? 0 : cy + 1;
        constexpr int CH = 16 / sizeof(T);  // reals per 16-byte chunk
#pragma unroll
        for (int k = 0; k < STAGE_SLOTS; k++) {
            const StageEntry e = stage_entry(k);
            const int x = e.dx < 0 ? xm : (e.dx > 0 ? xp : cx), y = e.dy < 0 ? ym : (e.dy > 0 ? yp : cy);
            const T* src = (e.b ? A.fn : A.fo) + fidx(8 * e.g, (size_t)x + (size_t)n * y, ns);
#pragma unroll
            for (int c = 0; c < 8; c += CH) cp_async16(rec + 8 * k + c, src + c);
        }
        cp_async_wait_all();
        const StagedSrc<T> F{rec};
        push_one_src<T, StagedSrc<T>>(A, F, j, sx, sy, sz, sc);
    }
    block_acc4(sx, sy, sz, sc, A.acc);
}

// ---------------------------------------------------------------- counting sort by cell
template <class T>
__global__ void k_scatter(PartSoA<T> a, PartSoA<T> b, int np, int* __restrict__ cursor) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int c = a.cell[j];
    const int k = atomicAdd(cursor + c, 1);
    b.cell[k] = c; b.pid[k] = a.pid[j];
    b.ox[k] = a.ox[j]; b.oy[k] = a.oy[j]; b.eta[k] = a.eta[j];
    b.p0x[k] = a.p0x[j]; b.p0y[k] = a.p0y[j]; b.p0z[k] = a.p0z[j];
    b.dpx[k] = a.dpx[j]; b.dpy[k] = a.dpy[j]; b.peta[k] = a.peta[j];
#pragma unroll
    for (int q = 0; q < 8; q++) b.Q[(size_t)q * b.qs + k] = a.Q[(size_t)q * a.qs + j];
}

}  // namespace glasma
