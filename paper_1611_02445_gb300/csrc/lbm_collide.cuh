// lbm_collide.cuh -- the local collision of one node (Eq. 2, 3, 7 with Guo forcing) in
// the arithmetic of the FP64-native, FP32 and FP16 storage formats, and the stochastic
// rounding of stores. Shared by the step kernels.
#pragma once
#include "lbm_internal.cuh"
#include "lbm_store.cuh"

namespace lbm {

// LBGK + Guo update of one direction pair (i, inv(i)) with lattice velocity c = c_i.
// Works on f (SHIFT = false, D = rho) or on h = f - w (SHIFT = true, D = rho - 1):
//   f^eq_i - w_i (if shifted) = w (D + rho (3 cu + 4.5 cu^2 - 1.5 u.u))      (Eq. 3)
//   S_i = beta w (3 (c - u).F + 9 (c.u)(c.F))                               (Guo)
//   v*_i = (1 - omega) v_i + omega v^eq_i + S_i                              (Eq. 7)
// split into the parts even (E, Se) and odd (O, So) in c.
template <typename R>
__device__ __forceinline__ void bgk_pair(R& a, R& b, R w, R cu, R cF, R D, R rho, R uu15, R uF3,
                                         R omega, R om1, R beta) {
    const R E = w * D + (w * rho) * (R(4.5) * cu * cu - uu15);
    const R O = R(3) * (w * rho) * cu;
    const R bw = beta * w;
    const R Se = bw * (R(9) * cu * cF - uF3);
    const R So = R(3) * bw * cF;
    a = om1 * a + (omega * (E + O) + (Se + So));
    b = om1 * b + (omega * (E - O) + (Se - So));
}

// The same update on h = f - w written with j' = rho u = j + F/2 (SHIFT = true):
//   h^eq_i = w (D + 3 c.j' + (4.5 (c.j')^2 - 1.5 |j'|^2) / rho),  D = rho - 1.
// The odd part 3 w c.j' then carries the momentum exactly as summed, instead of through
// the rounded u = j' / rho; the second-order part and the Guo term use 1 / rho.
//
// FP32 lattice constants: the collision conserves mass and momentum through two lattice
// identities, sum_i w_i = 1 (for w_i D) and sum_i 3 w_i c_ix^2 = 1 (for the odd part
// 3 w_i c_i.j'). With 1/3, 1/18, 1/36 rounded to FP32 the second is off by 3.0e-8, so
// every collision would add 3e-8 omega j' of momentum: a force proportional to the local
// velocity, a relative velocity error of ~3e-8 omega u / F in a slow steady flow. These
// constants satisfy both identities exactly in binary arithmetic (w1 = 14913080 2^-28,
// w2 = w1 / 2, w0 = 1 - 6 w1 - 12 w2 = 11184812 2^-25; a_k replaces 3 w_k in the odd
// part with 2 a1 + 8 a2 = 1: a1 = 11184810 2^-26, a2 = 11184811 2^-27) and differ from
// the exact weights by less than 2e-7 relative.
constexpr float W0S = 11184812.0f / 33554432.0f;
constexpr float W1S = 14913080.0f / 268435456.0f;
constexpr float W2S = 7456540.0f / 268435456.0f;
constexpr float A1S = 11184810.0f / 67108864.0f;
constexpr float A2S = 11184811.0f / 134217728.0f;

template <typename R>
__device__ __forceinline__ void bgk_pair_j(R& a, R& b, R w, R aw, R cj, R cF, R D, R inv_rho, R jj15, R uF3,
                                           R omega, R om1, R beta) {
    const R cu = cj * inv_rho;
    const R E = w * D + w * ((R(4.5) * cj * cj - jj15) * inv_rho);
    const R O = aw * cj;
    const R bw = beta * w;
    const R Se = bw * (R(9) * cu * cF - uF3);
    const R So = (beta * aw) * cF;
    a = om1 * a + (omega * (E + O) + (Se + So));
    b = om1 * b + (omega * (E - O) + (Se - So));
}

// Equilibrium of one direction pair: v_i = w (D + rho (3 cu + 4.5 cu^2 - 1.5 u.u)).
template <typename R>
__device__ __forceinline__ void eq_pair(R& a, R& b, R w, R cu, R D, R rho, R uu15) {
    const R E = w * D + (w * rho) * (R(4.5) * cu * cu - uu15);
    const R O = R(3) * (w * rho) * cu;
    a = E + O;
    b = E - O;
}

// Zou-He completion of an inlet (velocity u_in) or outlet (density rho_out, no tangential
// velocity) node on box face f = p.zh_face[0 or 1], inward normal n = +e_a (f = 2a) or
// -e_a (f = 2a + 1). The populations with c.n > 0 came from outside; with
// B = sum_{c.n=0} f + 2 sum_{c.n<0} f (1 + the same sums of h for the shifted formats,
// whose weights add up to 1 over these directions):
//   velocity: rho = B / (1 - u.n), j = rho u (Eq. 3 model); j = u, rho = B + u.n (Eq. 4);
//   pressure: j = (rho_out - B) n;
// then the unknown along n is f_opp + j_n / 3 and the unknown n + t e_b is
// f_opp + (j_n + t j_b) / 6 - t N_b, N_b = 1/2 sum_{c.n=0} c_b f - j_b / 3 (the transverse
// momentum correction of the D3Q19 form), so that the node has density rho and momentum j.
template <typename R, bool SHIFT>
__device__ __forceinline__ void zou_he(R v[Q], int type, const StepParams& p) {
    const int face = type == LBM_INLET ? p.zh_face[0] : p.zh_face[1];
    const int a = face >> 1;
    const int sg = (face & 1) ? -1 : 1;
    R B = SHIFT ? R(1) : R(0), T0 = 0, T1 = 0, T2 = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int cn = (a == 0 ? cx(i) : a == 1 ? cy(i) : cz(i)) * sg;
        if (cn == 0) {
            B += v[i];
            if (cx(i)) T0 += R(cx(i)) * v[i];
            if (cy(i)) T1 += R(cy(i)) * v[i];
            if (cz(i)) T2 += R(cz(i)) * v[i];
        } else if (cn < 0) {
            B += R(2) * v[i];
        }
    }
    R j0, j1, j2;
    if (type == LBM_INLET) {
        const R u0 = par<R>(p.u_in[0], p.u_in_f[0]), u1 = par<R>(p.u_in[1], p.u_in_f[1]),
                u2 = par<R>(p.u_in[2], p.u_in_f[2]);
        const R un = (a == 0 ? u0 : a == 1 ? u1 : u2) * R(sg);
        const bool inc = p.eq == LBM_EQ_INCOMPR;
        const R rho = inc ? B + un : B / (R(1) - un);
        const R s = inc ? R(1) : rho;
        j0 = s * u0;
        j1 = s * u1;
        j2 = s * u2;
    } else {
        const R jn = par<R>(p.rho_out, p.rho_out_f) - B;
        j0 = a == 0 ? jn * R(sg) : R(0);
        j1 = a == 1 ? jn * R(sg) : R(0);
        j2 = a == 2 ? jn * R(sg) : R(0);
    }
    const R jn = (a == 0 ? j0 : a == 1 ? j1 : j2) * R(sg);
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const int cn = (a == 0 ? cx(i) : a == 1 ? cy(i) : cz(i)) * sg;
        if (cn <= 0) continue;
        // tangential component of c_i, if any
        int b = -1, t = 0;
        if (a != 0 && cx(i) != 0) { b = 0; t = cx(i); }
        if (a != 1 && cy(i) != 0) { b = 1; t = cy(i); }
        if (a != 2 && cz(i) != 0) { b = 2; t = cz(i); }
        R val = v[inv(i)];
        if (b < 0) {
            val += jn * R(1.0 / 3.0);
        } else {
            const R jb = b == 0 ? j0 : b == 1 ? j1 : j2;
            const R Tb = b == 0 ? T0 : b == 1 ? T1 : T2;
            const R N = R(0.5) * Tb - jb * R(1.0 / 3.0);
            val += (jn + R(t) * jb) * R(1.0 / 6.0) - R(t) * N;
        }
        v[i] = val;
    }
}

// One node's collision, in place on v[19].
template <typename R, bool SHIFT>
__device__ __forceinline__ void collide(R v[Q], int type, const StepParams& p, R Fx, R Fy, R Fz) {
    if (type != LBM_FLUID && p.bc == LBM_BC_ZOU_HE) {
        // Zou-He boundary node: complete the unknown populations, then collide as fluid
        zou_he<R, SHIFT>(v, type, p);
        type = LBM_FLUID;
    }
    // moments from pair sums s and differences d of opposite directions
    const R s13 = v[1] + v[3], s24 = v[2] + v[4], s56 = v[5] + v[6], s79 = v[7] + v[9], s810 = v[8] + v[10];
    const R s1114 = v[11] + v[14], s1213 = v[12] + v[13], s1518 = v[15] + v[18], s1617 = v[16] + v[17];
    const R d13 = v[1] - v[3], d24 = v[2] - v[4], d56 = v[5] - v[6], d79 = v[7] - v[9], d810 = v[8] - v[10];
    const R d1114 = v[11] - v[14], d1213 = v[12] - v[13], d1518 = v[15] - v[18], d1617 = v[16] - v[17];
    const R sum = ((v[0] + s13) + (s24 + s56)) + ((s79 + s810) + (s1114 + s1213)) + (s1518 + s1617);
    const R jx = ((d13 + d79) - d810) + (d1114 + d1213);
    const R jy = ((d24 + d79) + d810) + (d1518 + d1617);
    const R jz = ((d56 + d1114) - d1213) + (d1518 - d1617);
    R D, rho;
    if (SHIFT) {
        D = sum;
        rho = R(1) + D;
    } else {
        rho = sum;
        D = sum;
    }
    const R inv_rho = R(1) / rho;
    const R Jx = jx + R(0.5) * Fx, Jy = jy + R(0.5) * Fy, Jz = jz + R(0.5) * Fz;
    const R ux = Jx * inv_rho;
    const R uy = Jy * inv_rho;
    const R uz = Jz * inv_rho;
    const R w0 = R(wgt(0)), w1 = R(wgt(1)), w2 = R(wgt(7));
    if (SHIFT && type == LBM_FLUID) {
        const R omega = par<R>(p.omega, p.omega_f), om1 = R(1) - omega, beta = par<R>(p.beta, p.beta_f);
        const R jj15 = R(1.5) * (Jx * Jx + Jy * Jy + Jz * Jz);
        const R uF3 = R(3) * (ux * Fx + uy * Fy + uz * Fz);
        const R s0 = R(W0S), s1 = R(W1S), s2 = R(W2S), a1 = R(A1S), a2 = R(A2S);
        v[0] = om1 * v[0] + (omega * (s0 * D - s0 * (jj15 * inv_rho)) - (beta * s0) * uF3);
        bgk_pair_j(v[1], v[3], s1, a1, Jx, Fx, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[2], v[4], s1, a1, Jy, Fy, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[5], v[6], s1, a1, Jz, Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[7], v[9], s2, a2, Jx + Jy, Fx + Fy, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[8], v[10], s2, a2, Jy - Jx, Fy - Fx, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[11], v[14], s2, a2, Jx + Jz, Fx + Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[12], v[13], s2, a2, Jx - Jz, Fx - Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[15], v[18], s2, a2, Jy + Jz, Fy + Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
        bgk_pair_j(v[16], v[17], s2, a2, Jy - Jz, Fy - Fz, D, inv_rho, jj15, uF3, omega, om1, beta);
    } else if (type == LBM_FLUID) {
        const R omega = par<R>(p.omega, p.omega_f), om1 = R(1) - omega, beta = par<R>(p.beta, p.beta_f);
        const R uu15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
        const R uF3 = R(3) * (ux * Fx + uy * Fy + uz * Fz);
        v[0] = om1 * v[0] + (omega * (w0 * D - (w0 * rho) * uu15) - (beta * w0) * uF3);
        bgk_pair(v[1], v[3], w1, ux, Fx, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[2], v[4], w1, uy, Fy, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[5], v[6], w1, uz, Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[7], v[9], w2, ux + uy, Fx + Fy, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[8], v[10], w2, uy - ux, Fy - Fx, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[11], v[14], w2, ux + uz, Fx + Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[12], v[13], w2, ux - uz, Fx - Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[15], v[18], w2, uy + uz, Fy + Fz, D, rho, uu15, uF3, omega, om1, beta);
        bgk_pair(v[16], v[17], w2, uy - uz, Fy - Fz, D, rho, uu15, uF3, omega, om1, beta);
    } else {
        // inlet: f^eq(rho, u_in); outlet: f^eq(rho_out, u)
        R ex, ey, ez, Dq, rq;
        if (type == LBM_INLET) {
            ex = par<R>(p.u_in[0], p.u_in_f[0]);
            ey = par<R>(p.u_in[1], p.u_in_f[1]);
            ez = par<R>(p.u_in[2], p.u_in_f[2]);
            Dq = D; rq = rho;
        } else {
            ex = ux; ey = uy; ez = uz;
            rq = par<R>(p.rho_out, p.rho_out_f);
            Dq = SHIFT ? par<R>(p.rho_out - 1.0, p.rho_out_m1_f) : rq;
        }
        const R uu15 = R(1.5) * (ex * ex + ey * ey + ez * ez);
        v[0] = w0 * Dq - (w0 * rq) * uu15;
        eq_pair(v[1], v[3], w1, ex, Dq, rq, uu15);
        eq_pair(v[2], v[4], w1, ey, Dq, rq, uu15);
        eq_pair(v[5], v[6], w1, ez, Dq, rq, uu15);
        eq_pair(v[7], v[9], w2, ex + ey, Dq, rq, uu15);
        eq_pair(v[8], v[10], w2, ey - ex, Dq, rq, uu15);
        eq_pair(v[11], v[14], w2, ex + ez, Dq, rq, uu15);
        eq_pair(v[12], v[13], w2, ex - ez, Dq, rq, uu15);
        eq_pair(v[15], v[18], w2, ey + ez, Dq, rq, uu15);
        eq_pair(v[16], v[17], w2, ey - ez, Dq, rq, uu15);
    }
}

// ------------------------------------------------------------------- other models
// D3Q19 moment basis of d'Humieres, Ginzburg, Krafczyk, Lallemand and Luo (2002): row k is
// a polynomial in the velocity c evaluated on the 19 lattice velocities; every entry is an
// integer. Rows: rho; e = 19|c|^2 - 30; eps = (21|c|^4 - 53|c|^2 + 24)/2; j_x; q_x = (5|c|^2 -
// 9) c_x; j_y; q_y; j_z; q_z; 3p_xx = 3c_x^2 - |c|^2; 3pi_xx = (3|c|^2 - 5) 3p_xx; p_ww =
// c_y^2 - c_z^2; pi_ww = (3|c|^2 - 5) p_ww; p_xy; p_yz; p_xz; m_x = (c_y^2 - c_z^2) c_x;
// m_y = (c_z^2 - c_x^2) c_y; m_z = (c_x^2 - c_y^2) c_z.
__host__ __device__ constexpr int mrt_row(int k, int i) {
    const int x = cx(i), y = cy(i), z = cz(i), cc = x * x + y * y + z * z;
    return k == 0 ? 1
         : k == 1 ? 19 * cc - 30
         : k == 2 ? (21 * cc * cc - 53 * cc + 24) / 2
         : k == 3 ? x : k == 4 ? (5 * cc - 9) * x
         : k == 5 ? y : k == 6 ? (5 * cc - 9) * y
         : k == 7 ? z : k == 8 ? (5 * cc - 9) * z
         : k == 9 ? 3 * x * x - cc
         : k == 10 ? (3 * cc - 5) * (3 * x * x - cc)
         : k == 11 ? y * y - z * z
         : k == 12 ? (3 * cc - 5) * (y * y - z * z)
         : k == 13 ? x * y : k == 14 ? y * z : k == 15 ? x * z
         : k == 16 ? (y * y - z * z) * x
         : k == 17 ? (z * z - x * x) * y
         : (x * x - y * y) * z;
}
__host__ __device__ constexpr int mrt_norm(int k) {
    int n = 0;
    for (int i = 0; i < Q; i++) n += mrt_row(k, i) * mrt_row(k, i);
    return n;
}

// Equilibrium of model eq at (rq, u), as f (SHIFT = false; Dq = rq) or as h = f - w
// (SHIFT = true; Dq = rq - 1): w (Dq + a (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)) with a = rq for the
// quasi-compressible Eq. 3 and a = 1 for the incompressible Eq. 4.
template <typename R>
__device__ __forceinline__ R feq_model(int i, R Dq, R a, R ex, R ey, R ez, R uu15) {
    const R cu = R(cx(i)) * ex + R(cy(i)) * ey + R(cz(i)) * ez;
    return R(wgt(i)) * (Dq + a * (R(3) * cu + R(4.5) * cu * cu - uu15));
}

// Collision of one node for the models other than quasi-compressible LBGK: the
// incompressible equilibrium (Eq. 4, velocity Eq. 6: u = j + F/2) and MRT (Eq. 8):
//   m = M (v - v^eq), mG = M G, v* = v^eq + M^T (mrt_a . m + mrt_b . mG),
// G_i = w_i (3 (c_i - u).F + 9 (c_i.u)(c_i.F)) (Guo forcing in moment space); LBGK is
//   v* = (1 - omega) v + omega v^eq + (1 - omega/2) G.
template <typename R, bool SHIFT>
__device__ __forceinline__ void collide_model(R v[Q], int type, const StepParams& p, R Fx, R Fy, R Fz) {
    if (type != LBM_FLUID && p.bc == LBM_BC_ZOU_HE) {
        zou_he<R, SHIFT>(v, type, p);
        type = LBM_FLUID;
    }
    R sum = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        sum += v[i];
        if (cx(i)) jx += R(cx(i)) * v[i];
        if (cy(i)) jy += R(cy(i)) * v[i];
        if (cz(i)) jz += R(cz(i)) * v[i];
    }
    const R rho = SHIFT ? R(1) + sum : sum;
    const R D = sum;
    const bool inc = p.eq == LBM_EQ_INCOMPR;
    const R Jx = jx + R(0.5) * Fx, Jy = jy + R(0.5) * Fy, Jz = jz + R(0.5) * Fz;
    const R ir = inc ? R(1) : R(1) / rho;
    const R ux = Jx * ir, uy = Jy * ir, uz = Jz * ir;
    if (type == LBM_INLET || type == LBM_OUTLET) {
        R ex, ey, ez, Dq, rq;
        if (type == LBM_INLET) {
            ex = par<R>(p.u_in[0], p.u_in_f[0]);
            ey = par<R>(p.u_in[1], p.u_in_f[1]);
            ez = par<R>(p.u_in[2], p.u_in_f[2]);
            Dq = D;
            rq = rho;
        } else {
            ex = ux; ey = uy; ez = uz;
            rq = par<R>(p.rho_out, p.rho_out_f);
            Dq = SHIFT ? par<R>(p.rho_out - 1.0, p.rho_out_m1_f) : rq;
        }
        const R uu15 = R(1.5) * (ex * ex + ey * ey + ez * ez);
        const R a = inc ? R(1) : rq;
#pragma unroll
        for (int i = 0; i < Q; i++) v[i] = feq_model<R>(i, Dq, a, ex, ey, ez, uu15);
        return;
    }
    const R uu15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
    const R a = inc ? R(1) : rho;
    const R uF3 = R(3) * (ux * Fx + uy * Fy + uz * Fz);
    R ve[Q], G[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        ve[i] = feq_model<R>(i, D, a, ux, uy, uz, uu15);
        const R cu = R(cx(i)) * ux + R(cy(i)) * uy + R(cz(i)) * uz;
        const R cF = R(cx(i)) * Fx + R(cy(i)) * Fy + R(cz(i)) * Fz;
        G[i] = R(wgt(i)) * (R(3) * cF - uF3 + R(9) * cu * cF);
    }
    if (p.coll == LBM_COLL_BGK) {
        const R omega = par<R>(p.omega, p.omega_f), beta = par<R>(p.beta, p.beta_f);
#pragma unroll
        for (int i = 0; i < Q; i++) v[i] = v[i] + omega * (ve[i] - v[i]) + beta * G[i];
        return;
    }
    R ms[Q];
#pragma unroll
    for (int k = 0; k < Q; k++) {
        R md = 0, mg = 0;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            if (mrt_row(k, i) != 0) {
                md += R(mrt_row(k, i)) * (v[i] - ve[i]);
                mg += R(mrt_row(k, i)) * G[i];
            }
        }
        ms[k] = par<R>(p.mrt_a[k], p.mrt_a_f[k]) * md + par<R>(p.mrt_b[k], p.mrt_b_f[k]) * mg;
    }
#pragma unroll
    for (int i = 0; i < Q; i++) {
        R acc = ve[i];
#pragma unroll
        for (int k = 0; k < Q; k++)
            if (mrt_row(k, i) != 0) acc += R(mrt_row(k, i)) * ms[k];
        v[i] = acc;
    }
}

// ------------------------------------------------------------ stochastic rounding
// MurmurHash3's 32-bit finaliser (A. Appleby, public domain): a bijective avalanche mix,
// used as a counter-based generator keyed by (step counter, node, direction pair).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// binary16 nearest to x + d, d = (r - 32767.5) 2^-16 s uniform over one binary16 spacing
// s of x (r: 16 random bits). For x in (lo, lo + s) this rounds up with probability
// (x - lo) / s to 16 bits, i.e. stochastic rounding (the FP32 sum x + d is off by at most
// 2^-14 s). s = 2^(e - 10) for |x| >= 2^-14 (e the exponent of x), 2^-24 below.
__device__ __forceinline__ __half half_dithered(float x, uint32_t r) {
    const uint32_t eb = __float_as_uint(x) & 0x7f800000u;
    const uint32_t sb = max(eb, 113u << 23) - (26u << 23);   // s * 2^-16
    const float d = __fmul_rn(__int2float_rn((int)r - 32767) - 0.5f, __uint_as_float(sb));
    return __float2half_rn(__fadd_rn(x, d));
}

}  // namespace lbm
