// lbm_collide_df.cuh -- LBGK + Guo collision of a fluid node with FP64 inputs and outputs
// and double-float arithmetic in between.
//
// GB300 executes FP64 on 2 lanes per SM and clock against 128 for FP32, so the FP64
// storage path spends one FP64 instruction per population, the fused multiply-add at
// the end, plus four per node for the dominant term omega w rho; the moment sums rho, j
// are exact 64-bit integer sums of the stored doubles in fixed point (2^-58), formed
// from their bit patterns:
//     f*_i = (1 - omega) f_i + Y_i,   Y_i = omega f^eq_i + S_i          (Eq. 2, 3, 7; Guo)
// Y_i is formed in double-float (about 48 bits). With rho u = j' = j + F/2:
//     omega f^eq_i = omega w (rho + 3 c.j' + Q_i),  Q_i = (4.5 (c.j')^2 - 1.5 |j'|^2) / rho,
//     S_i = beta w (3 c.F - 3 u.F + 9 (c.u)(c.F)),
// split per direction pair into the parts even in c,
//     Ye = omega w (rho + Q) + 9 beta w (c.u)(c.F) - 3 beta w (u.F),
// and odd in c, Yo = 3 omega w (c.j') + 3 beta w (c.F); Y_i = Ye + Yo, Y_inv(i) = Ye - Yo.
#pragma once
#include "lbm_df.cuh"

namespace lbm {

// Per-launch constants, computed on the host in FP64 and split into pairs; class 0 is
// the rest weight 1/3, class 1 the axis weight 1/18, class 2 the diagonal weight 1/36.
struct DFConst {
    double om1;          // 1 - omega
    dfl ow[3];           // omega w
    double ow_d[3];      // omega w in FP64, for the dominant term omega w rho
    dfl ow3[3];          // 3 omega w
    dfl bw[3];           // beta w
    dfl bw3[3];          // 3 beta w
    dfl bw9[3];          // 9 beta w
    dfl Fy, Fz;          // uniform y, z force density
    double Fy_d, Fz_d;   // the same in FP64
};

LBM_DF_HD dfl df_split_host(double v) {
    const float h = (float)v;
    return df_make(h, (float)(v - (double)h));
}

LBM_DF_HD DFConst make_df_const(double omega, double beta, double Fy, double Fz) {
    DFConst c;
    const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    c.om1 = 1.0 - omega;
    for (int k = 0; k < 3; k++) {
        c.ow[k] = df_split_host(omega * w[k]);
        c.ow_d[k] = omega * w[k];
        c.ow3[k] = df_split_host(3.0 * omega * w[k]);
        c.bw[k] = df_split_host(beta * w[k]);
        c.bw3[k] = df_split_host(3.0 * beta * w[k]);
        c.bw9[k] = df_split_host(9.0 * beta * w[k]);
    }
    c.Fy = df_split_host(Fy);
    c.Fz = df_split_host(Fz);
    c.Fy_d = Fy;
    c.Fz_d = Fz;
    return c;
}

// One direction pair (a with velocity c, b with -c) of weight class k.
LBM_DF_HD void df_pair(double& a, double& b, const DFConst& K, int k, dfl cj, dfl cF, dfl inv, dfl A, dfl Gu,
                       dfl JJ15) {
    const dfl cu = df_mul(cj, inv);
    const dfl Q = df_mul(df_sub(df_mulf(df_mul(cj, cj), 4.5f), JJ15), inv);
    const dfl Ye = df_sub(df_add(df_add(A, df_mul(K.ow[k], Q)), df_mul(K.bw9[k], df_mul(cu, cF))), Gu);
    const dfl Yo = df_add(df_mul(K.ow3[k], cj), df_mul(K.bw3[k], cF));
    const double yp = df_to_double_pos(df_add(Ye, Yo));
    const double ym = df_to_double_pos(df_sub(Ye, Yo));
#if defined(__CUDA_ARCH__)
    a = __fma_rn(K.om1, a, yp);
    b = __fma_rn(K.om1, b, ym);
#else
    a = std::fma(K.om1, a, yp);
    b = std::fma(K.om1, b, ym);
#endif
}

// f: the 19 gathered populations of a fluid node, replaced by the post-collision ones.
LBM_DF_HD void collide_df(double f[19], double Fx, const DFConst& K) {
    // exact moments in 64-bit fixed point, from pair sums s and differences d of
    // opposite directions (the FP64 pipe is kept for the final update)
    int64_t q[19];
#pragma unroll
    for (int i = 0; i < 19; i++) q[i] = fix_from_double(f[i]);
    const int64_t s13 = q[1] + q[3], s24 = q[2] + q[4], s56 = q[5] + q[6], s79 = q[7] + q[9], s810 = q[8] + q[10];
    const int64_t s1114 = q[11] + q[14], s1213 = q[12] + q[13], s1518 = q[15] + q[18], s1617 = q[16] + q[17];
    const int64_t d13 = q[1] - q[3], d24 = q[2] - q[4], d56 = q[5] - q[6], d79 = q[7] - q[9], d810 = q[8] - q[10];
    const int64_t d1114 = q[11] - q[14], d1213 = q[12] - q[13], d1518 = q[15] - q[18], d1617 = q[16] - q[17];
    const int64_t rho = q[0] + s13 + s24 + s56 + s79 + s810 + s1114 + s1213 + s1518 + s1617;
    const int64_t jx = d13 + d79 - d810 + d1114 + d1213;
    const int64_t jy = d24 + d79 + d810 + d1518 + d1617;
    const int64_t jz = d56 + d1114 - d1213 + d1518 - d1617;
    // j' = j + F/2 (F/2 in the same fixed point, truncated: |error| < 2^-58)
    const dfl Jx = df_from_fix(jx + (fix_from_double(Fx) >> 1));
    const dfl Jy = df_from_fix(jy + (fix_from_double(K.Fy_d) >> 1));
    const dfl Jz = df_from_fix(jz + (fix_from_double(K.Fz_d) >> 1));
    const dfl R = df_from_fix(rho);
    const dfl inv = df_recip(R);
    const dfl ux = df_mul(Jx, inv), uy = df_mul(Jy, inv), uz = df_mul(Jz, inv);
    const dfl Fxd = df_from_double(Fx);
    const dfl JJ15 = df_mulf(df_add(df_add(df_mul(Jx, Jx), df_mul(Jy, Jy)), df_mul(Jz, Jz)), 1.5f);
    const dfl uF3 = df_mulf(df_add(df_add(df_mul(ux, Fxd), df_mul(uy, K.Fy)), df_mul(uz, K.Fz)), 3.0f);
    dfl A[3], Gu[3];
#pragma unroll
    // omega w rho dominates every Y_i, so it is formed in FP64 (one conversion and three
    // multiplies per node): a double-float product with a rounded constant would leave a
    // systematic relative bias of ~1e-15 that acts as a mass source
#if defined(__CUDA_ARCH__)
    const double rho_d = __dmul_rn(__ll2double_rn(rho), 1.0 / (double)(1ull << FIX_SHIFT));
#else
    const double rho_d = (double)rho * (1.0 / (double)(1ull << FIX_SHIFT));
#endif
    for (int k = 0; k < 3; k++) {
        A[k] = df_from_double(K.ow_d[k] * rho_d);
        Gu[k] = df_mul(K.bw[k], uF3);
    }
    // rest population: Y0 = omega w0 (rho - 1.5 |j'|^2 / rho) - 3 beta w0 (u.F)
    const dfl Y0 = df_sub(df_sub(A[0], df_mul(K.ow[0], df_mul(JJ15, inv))), Gu[0]);
#if defined(__CUDA_ARCH__)
    f[0] = __fma_rn(K.om1, f[0], df_to_double_pos(Y0));
#else
    f[0] = std::fma(K.om1, f[0], df_to_double_pos(Y0));
#endif
    df_pair(f[1], f[3], K, 1, Jx, Fxd, inv, A[1], Gu[1], JJ15);
    df_pair(f[2], f[4], K, 1, Jy, K.Fy, inv, A[1], Gu[1], JJ15);
    df_pair(f[5], f[6], K, 1, Jz, K.Fz, inv, A[1], Gu[1], JJ15);
    df_pair(f[7], f[9], K, 2, df_add(Jx, Jy), df_add(Fxd, K.Fy), inv, A[2], Gu[2], JJ15);
    df_pair(f[8], f[10], K, 2, df_sub(Jy, Jx), df_sub(K.Fy, Fxd), inv, A[2], Gu[2], JJ15);
    df_pair(f[11], f[14], K, 2, df_add(Jx, Jz), df_add(Fxd, K.Fz), inv, A[2], Gu[2], JJ15);
    df_pair(f[12], f[13], K, 2, df_sub(Jx, Jz), df_sub(Fxd, K.Fz), inv, A[2], Gu[2], JJ15);
    df_pair(f[15], f[18], K, 2, df_add(Jy, Jz), df_add(K.Fy, K.Fz), inv, A[2], Gu[2], JJ15);
    df_pair(f[16], f[17], K, 2, df_sub(Jy, Jz), df_sub(K.Fy, K.Fz), inv, A[2], Gu[2], JJ15);
}

}  // namespace lbm
