// lbm_collide_df.cuh -- LBGK + Guo collision of a fluid node with FP64 inputs and outputs
// and double-float arithmetic in between.
//
// GB300 executes FP64 on 2 lanes per SM and clock against 128 for FP32, so the FP64
// storage path spends one FP64 instruction per population, the fused multiply-add at
// the end, plus three per node for the dominant term omega w rho; the moment sums rho, j
// are exact 64-bit integer sums of the stored doubles in fixed point (2^-58), formed
// from their bit patterns:
//     f*_i = (1 - omega) f_i + Y_i,   Y_i = omega f^eq_i + S_i          (Eq. 2, 3, 7; Guo)
// Y_i is formed in double-float (about 48 bits). With rho u = j' = j + F/2:
//     omega f^eq_i = omega w (rho + 3 c.j' + Q_i),  Q_i = (4.5 (c.j')^2 - 1.5 |j'|^2) / rho,
//     S_i = beta w (3 c.F - 3 u.F + 9 (c.u)(c.F)),
// split per direction pair into the parts even in c,
//     Ye = omega w rho - (w / rho) P + (w / rho) c.j' (4.5 omega c.j' + 9 beta c.F),
//     P  = 1.5 omega |j'|^2 + 3 beta j'.F   (once per node),
// and odd in c, Yo = 3 omega w (c.j') + 3 beta w (c.F); Y_i = Ye + Yo, Y_inv(i) = Ye - Yo.
// Since 4.5 omega w = 1.5 (3 omega w) and 9 beta w = 1.5 (2 * 3 beta w), the last term of
// Ye is (1.5 / rho) c.j' (Yo + 3 beta w c.F): it reuses Yo, and the even part needs one
// product with c.j' and one with 1.5 / rho per pair.
#pragma once
#include "lbm_df.cuh"

namespace lbm {

// Per-launch constants, computed on the host in FP64 and split into pairs; class 0 is
// the rest weight 1/3, class 1 the axis weight 1/18, class 2 the diagonal weight 1/36.
struct DFConst {
    double om1;          // 1 - omega
    double ow_d[2];      // omega w0 2^-58, omega w1 2^-58 in FP64: the dominant term omega w rho
                         // from the fixed-point density (w2 = w1 / 2 exactly, so omega w2 rho
                         // is the class-1 product halved)
    dfl ow3[3];          // 3 omega w
    dfl om15;            // 1.5 omega
    dfl b3;              // 3 beta
    dfl w0, w1;          // 1/3, 1/18
    dfl bw3;             // 3 beta w1
    dfl Fy, Fz;          // uniform y, z force density
    dfl G3y, G3z;        // 3 beta w1 F_y, 3 beta w1 F_z
    int64_t Fy2q, Fz2q;  // F_y / 2, F_z / 2 in 2^-58 fixed point (truncated)
    // The uniform x force (g[0]) and its terms, used when no per-node force field is set:
    // F_x / 2 in fixed point, F_x and 3 beta w1 F_x.
    int64_t Fx2q;
    dfl Fx, G3x;
};

// 3 beta w c.F of direction pair k of (1,3) (2,4) (5,6) (7,9) (8,10) (11,14) (12,13)
// (15,18) (16,17) from the per-axis terms G3 = 3 beta w1 F: a diagonal pair's is half the
// sum or difference of its axes' (w2 = w1 / 2). k is a constant after unrolling, so the
// switch folds away.
LBM_DF_HD dfl df_g3(int k, dfl G3x, dfl G3y, dfl G3z) {
    switch (k) {
        case 0: return G3x;
        case 1: return G3y;
        case 2: return G3z;
        case 3: return df_scale2(df_add(G3x, G3y), 0.5f);
        case 4: return df_scale2(df_sub(G3y, G3x), 0.5f);
        case 5: return df_scale2(df_add(G3x, G3z), 0.5f);
        case 6: return df_scale2(df_sub(G3x, G3z), 0.5f);
        case 7: return df_scale2(df_add(G3y, G3z), 0.5f);
        default: return df_scale2(df_sub(G3y, G3z), 0.5f);
    }
}

// The same for a force along x alone: pairs 0 (1,3), 3 (7,9), 5 (11,14) and 6 (12,13) have
// c_x = +1 on their first direction, pair 4 (8,10) has c_x = -1; the others have c_x = 0
// and no force terms. 3 beta w c.F is G3x for the axis pair and +-G3x / 2 (`half`) for a
// diagonal one.
LBM_DF_HD bool df_pair_has_fx(int k) { return k == 0 || (k >= 3 && k <= 6); }
LBM_DF_HD dfl df_pair_g3x(int k, dfl G3x, dfl half) {
    return k == 0 ? G3x : k == 4 ? df_make(-half.h, -half.l) : half;
}

LBM_DF_HD dfl df_split_host(double v) {
    const float h = (float)v;
    return df_make(h, (float)(v - (double)h));
}

LBM_DF_HD DFConst make_df_const(double omega, double beta, double Fx, double Fy, double Fz) {
    DFConst c;
    const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    c.om1 = 1.0 - omega;
    for (int k = 0; k < 3; k++) {
        if (k < 2) c.ow_d[k] = omega * w[k] * (1.0 / (double)(1ull << FIX_SHIFT));   // exact scaling
        c.ow3[k] = df_split_host(3.0 * omega * w[k]);
    }
    c.om15 = df_split_host(1.5 * omega);
    c.b3 = df_split_host(3.0 * beta);
    c.w0 = df_split_host(w[0]);
    c.w1 = df_split_host(w[1]);
    c.bw3 = df_split_host(3.0 * beta * w[1]);
    c.Fy = df_split_host(Fy);
    c.Fz = df_split_host(Fz);
    c.G3y = df_split_host(3.0 * beta * w[1] * Fy);
    c.G3z = df_split_host(3.0 * beta * w[1] * Fz);
    c.Fy2q = fix_from_double(Fy) >> 1;
    c.Fz2q = fix_from_double(Fz) >> 1;
    c.Fx2q = fix_from_double(Fx) >> 1;
    c.Fx = df_split_host(Fx);
    c.G3x = df_split_host(3.0 * beta * w[1] * Fx);
    return c;
}

// Per-launch constants of the equilibrium closures of inlet and outlet nodes (the boundary
// scheme LBM_BC_EQUILIBRIUM): an inlet node takes f^eq(rho, u_in) from its own density,
// i.e. rho times kin_i = w_i (1 + 3 c.u_in + 4.5 (c.u_in)^2 - 1.5 |u_in|^2), held here with
// the 2^-58 of the fixed-point density folded in; an outlet node takes f^eq(rho_out, u)
// with its own velocity, whose weights w rho_out come per class, in pairs.
struct DFClosure {
    double kin[19];
    dfl wout[3], w3out[3];   // w rho_out, 3 w rho_out
};

LBM_DF_HD DFClosure make_df_closure(const double u_in[3], double rho_out) {
    // D3Q19 velocities in the library's numbering: 0 rest; 1 E 2 N 3 W 4 S 5 T 6 B;
    // 7 NE 8 NW 9 SW 10 SE; 11 ET 12 EB 13 WT 14 WB; 15 NT 16 NB 17 ST 18 SB
    const int c[19][3] = {{0, 0, 0},   {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                          {1, 1, 0},   {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {1, 0, 1},  {1, 0, -1}, {-1, 0, 1},
                          {-1, 0, -1}, {0, 1, 1},  {0, 1, -1},  {0, -1, 1}, {0, -1, -1}};
    const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    const double uu = u_in[0] * u_in[0] + u_in[1] * u_in[1] + u_in[2] * u_in[2];
    DFClosure b;
    for (int i = 0; i < 19; i++) {
        const double cu = c[i][0] * u_in[0] + c[i][1] * u_in[1] + c[i][2] * u_in[2];
        const double wi = w[i == 0 ? 0 : i < 7 ? 1 : 2];
        b.kin[i] = wi * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu) * (1.0 / (double)(1ull << FIX_SHIFT));
    }
    for (int k = 0; k < 3; k++) {
        b.wout[k] = df_split_host(w[k] * rho_out);
        b.w3out[k] = df_split_host(3.0 * w[k] * rho_out);
    }
    return b;
}

// One direction pair (a with velocity c, b with -c) of weight class k, with cj = c.j',
// g3 = 3 beta w c.F, AP = omega w rho - (w / rho) P (per weight class), r15 = 1.5 / rho:
//   Yo = 3 omega w cj + g3,   Ye = AP + r15 cj (Yo + g3).
// The even part dominates: |omega w rho| >= |w T / rho| and |Ye| >= |Yo| hold while
// |c.u| < 1/3 (T <= 9 omega j^2, Yo ~ 3 omega w rho c.u), far inside the low-Mach range
// of the method, so those three sums use FastTwoSum.
// has_f false: the pair's force term g3 is zero (c.F = 0) and its sums are left out.
LBM_DF_HD void df_pair(double& a, double& b, const DFConst& K, int k, dfl cj, bool has_f, dfl g3, dfl r15, dfl AP) {
    const dfl o = df_mul(K.ow3[k], cj);
    const dfl Yo = has_f ? df_add(o, g3) : o;
    const dfl Z = has_f ? df_add(Yo, g3) : Yo;
    const dfl Ye = df_add_dom(AP, df_mul(r15, df_mul(cj, Z)));
    const double yp = df_to_double_pos(df_add_dom(Ye, Yo));
    const double ym = df_to_double_pos(df_sub_dom(Ye, Yo));
#if defined(__CUDA_ARCH__)
    a = __fma_rn(K.om1, a, yp);
    b = __fma_rn(K.om1, b, ym);
#else
    a = std::fma(K.om1, a, yp);
    b = std::fma(K.om1, b, ym);
#endif
}

// Density and momentum from the 19 fixed-point populations, through the pair sums and
// differences of opposite directions.
LBM_DF_HD void fix_moments(const int64_t q[19], int64_t& rho, int64_t& jx, int64_t& jy, int64_t& jz) {
    const int64_t s13 = q[1] + q[3], s24 = q[2] + q[4], s56 = q[5] + q[6], s79 = q[7] + q[9], s810 = q[8] + q[10];
    const int64_t s1114 = q[11] + q[14], s1213 = q[12] + q[13], s1518 = q[15] + q[18], s1617 = q[16] + q[17];
    const int64_t d13 = q[1] - q[3], d24 = q[2] - q[4], d56 = q[5] - q[6], d79 = q[7] - q[9], d810 = q[8] - q[10];
    const int64_t d1114 = q[11] - q[14], d1213 = q[12] - q[13], d1518 = q[15] - q[18], d1617 = q[16] - q[17];
    rho = q[0] + s13 + s24 + s56 + s79 + s810 + s1114 + s1213 + s1518 + s1617;
    jx = d13 + d79 - d810 + d1114 + d1213;
    jy = d24 + d79 + d810 + d1518 + d1617;
    jz = d56 + d1114 - d1213 + d1518 - d1617;
}

// Exact moments of a node in 64-bit fixed point. Populations in [2^-6, 16), every one of a
// node near equilibrium at |u| below about 0.15, convert with six integer instructions
// each; a node with any other value (negative, smaller, larger) converts all 19 again on
// the FP64 pipe, which rounds the small ones to nearest. That fallback needs few
// registers; the general integer conversion in its place made the whole step 10 % slower.
LBM_DF_HD void node_moments(const double f[19], int64_t& rho, int64_t& jx, int64_t& jy, int64_t& jz) {
    int64_t q[19];
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 19; i++) q[i] = fix_from_double_fast(f[i], bad);
    fix_moments(q, rho, jx, jy, jz);
    if (bad) {
#pragma unroll
        for (int i = 0; i < 19; i++) q[i] = fix_from_double_cvt(f[i]);
        fix_moments(q, rho, jx, jy, jz);
    }
}

// f: the 19 gathered populations of a fluid node, replaced by the post-collision ones.
// uniform_fx: Fx is the uniform force K was built with, so every term that depends on it
// comes from K; otherwise (a per-node force field) they are formed here.
// XF: K was built with F_y = F_z = 0 (a force along x, or none), so the terms of F_y and
// F_z, and the force terms of the pairs with c_x = 0, are left out; with those inputs the
// results equal the general form's bit for bit (the omitted sums add exact zeros).
// INC: the incompressible equilibrium (Eq. 4, with u from Eq. 6 and the reference density
// 1 in place of rho): f^eq = w (rho + 3 c.j' + 4.5 (c.j')^2 - 1.5 |j'|^2) and the Guo term
// with u = j', which is the form above with 1 / rho replaced by 1.
template <bool XF, bool INC = false>
LBM_DF_HD void collide_df(double f[19], double Fx, const DFConst& K, bool uniform_fx) {
    int64_t rho, jx, jy, jz;
    node_moments(f, rho, jx, jy, jz);
    // j' = j + F/2 (F/2 in the same fixed point, truncated: |error| < 2^-58)
    const dfl Jx = df_from_fix(jx + (uniform_fx ? K.Fx2q : fix_from_double(Fx) >> 1));
    const dfl Jy = df_from_fix(XF ? jy : jy + K.Fy2q);
    const dfl Jz = df_from_fix(XF ? jz : jz + K.Fz2q);
    const dfl inv = INC ? df_make(1.0f, 0.0f) : df_recip(df_from_fix(rho));
    const dfl Fxd = uniform_fx ? K.Fx : df_from_double(Fx);
    // P = 1.5 omega |j'|^2 + 3 beta j'.F: the isotropic second-order part of every Y_i
    const dfl JJ = df_add(df_add(df_mul(Jx, Jx), df_mul(Jy, Jy)), df_mul(Jz, Jz));
    const dfl JF = XF ? df_mul(Jx, Fxd) : df_add(df_add(df_mul(Jx, Fxd), df_mul(Jy, K.Fy)), df_mul(Jz, K.Fz));
    const dfl P = df_add(df_mul(K.om15, JJ), df_mul(K.b3, JF));
    // omega w rho dominates every Y_i, so it is formed in FP64 (one conversion and two
    // multiplies per node): a double-float product with a rounded constant would leave a
    // systematic relative bias of ~1e-15 that acts as a mass source. The 2^-58 of the
    // fixed point sits in the constants, and omega w2 rho = (omega w1 rho) / 2 exactly.
#if defined(__CUDA_ARCH__)
    const double rho_i = __ll2double_rn(rho);
#else
    const double rho_i = (double)rho;
#endif
    // rest population: Y0 = A0 - (w0 / rho) P
    const dfl A0 = df_from_double(K.ow_d[0] * rho_i);
    const dfl Y0 = df_sub_dom(A0, df_mul(INC ? K.w0 : df_mul(K.w0, inv), P));   // |A0| dominates while |u|^2 < 2/3
#if defined(__CUDA_ARCH__)
    f[0] = __fma_rn(K.om1, f[0], df_to_double_pos(Y0));
#else
    f[0] = std::fma(K.om1, f[0], df_to_double_pos(Y0));
#endif
    // AP = omega w rho - (w / rho) P of the axis class, halved (exactly) for the diagonal one
    const dfl AP1 = df_sub_dom(df_from_double(K.ow_d[1] * rho_i), df_mul(INC ? K.w1 : df_mul(K.w1, inv), P));
    const dfl AP2 = df_scale2(AP1, 0.5f);
    const dfl r15 = INC ? df_make(1.5f, 0.0f) : df_mulf(inv, 1.5f);
    // 3 beta w1 F_x from K with a uniform force; with XF only the pairs with c_x != 0 carry
    // a force
    const dfl G3x = uniform_fx ? K.G3x : df_mul(K.bw3, Fxd);
#define LBM_DF_PAIR(a, b, cls, k, cj, AP)                                                                    \
    df_pair(f[a], f[b], K, cls, cj, !XF || df_pair_has_fx(k),                                                \
            XF ? df_pair_g3x(k, G3x, df_scale2(G3x, 0.5f)) : df_g3(k, G3x, K.G3y, K.G3z), r15, AP)
    LBM_DF_PAIR(1, 3, 1, 0, Jx, AP1);
    LBM_DF_PAIR(2, 4, 1, 1, Jy, AP1);
    LBM_DF_PAIR(5, 6, 1, 2, Jz, AP1);
    LBM_DF_PAIR(7, 9, 2, 3, df_add(Jx, Jy), AP2);
    LBM_DF_PAIR(8, 10, 2, 4, df_sub(Jy, Jx), AP2);
    LBM_DF_PAIR(11, 14, 2, 5, df_add(Jx, Jz), AP2);
    LBM_DF_PAIR(12, 13, 2, 6, df_sub(Jx, Jz), AP2);
    LBM_DF_PAIR(15, 18, 2, 7, df_add(Jy, Jz), AP2);
    LBM_DF_PAIR(16, 17, 2, 8, df_sub(Jy, Jz), AP2);
#undef LBM_DF_PAIR
}

// Equilibrium closure of an inlet (type 2) or outlet (type 3) node, replacing the 19
// gathered populations f: the inlet's f^eq(rho, u_in) is its exact density times the
// per-launch kin_i, one FP64 multiply per population; the outlet's f^eq(rho_out, u),
// u = (j + F/2) / rho, is formed in double-float like the collision's pairs,
//     f_a, f_b = E +- O,  E = w rho_out (1 - 1.5 |u|^2 + 4.5 (c.u)^2),  O = 3 w rho_out c.u,
// and widened to FP64 without an FP64 instruction. Both keep the closures off the FP64
// pipe's long dependent chains, which held the rest of a CTA at its per-group barrier.
LBM_DF_HD void closure_df(double f[19], int type, double Fx, const DFConst& K, const DFClosure& B, bool uniform_fx) {
    int64_t rho, jx, jy, jz;
    node_moments(f, rho, jx, jy, jz);
    if (type == 2) {   // LBM_INLET
#if defined(__CUDA_ARCH__)
        const double r = __ll2double_rn(rho);
#pragma unroll
        for (int i = 0; i < 19; i++) f[i] = __dmul_rn(r, B.kin[i]);
#else
        const double r = (double)rho;
        for (int i = 0; i < 19; i++) f[i] = r * B.kin[i];
#endif
        return;
    }
    const dfl inv = df_recip(df_from_fix(rho));
    const dfl ux = df_mul(df_from_fix(jx + (uniform_fx ? K.Fx2q : fix_from_double(Fx) >> 1)), inv);
    const dfl uy = df_mul(df_from_fix(jy + K.Fy2q), inv);
    const dfl uz = df_mul(df_from_fix(jz + K.Fz2q), inv);
    const dfl uu = df_add(df_add(df_mul(ux, ux), df_mul(uy, uy)), df_mul(uz, uz));
    const dfl E0 = df_add_dom(df_make(1.0f, 0.0f), df_mulf(uu, -1.5f));   // 1 - 1.5 |u|^2
    f[0] = df_to_double_pos(df_mul(B.wout[0], E0));
    auto pair = [&](double& a, double& b, int k, dfl cu) {
        const dfl E = df_mul(B.wout[k], df_add_dom(E0, df_mulf(df_mul(cu, cu), 4.5f)));
        const dfl O = df_mul(B.w3out[k], cu);
        a = df_to_double_pos(df_add_dom(E, O));
        b = df_to_double_pos(df_sub_dom(E, O));
    };
    pair(f[1], f[3], 1, ux);
    pair(f[2], f[4], 1, uy);
    pair(f[5], f[6], 1, uz);
    pair(f[7], f[9], 2, df_add(ux, uy));
    pair(f[8], f[10], 2, df_sub(uy, ux));
    pair(f[11], f[14], 2, df_add(ux, uz));
    pair(f[12], f[13], 2, df_sub(ux, uz));
    pair(f[15], f[18], 2, df_add(uy, uz));
    pair(f[16], f[17], 2, df_sub(uy, uz));
}

}  // namespace lbm
