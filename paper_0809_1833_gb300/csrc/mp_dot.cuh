// FP32 correlation <r, psi_m> (Eq. 9) with one fixed summation order, used
// by every kernel that computes a correlation in FP32 so that all launch
// shapes give the same bits.
#pragma once
#include "mp_device.cuh"

namespace mpgb {

// Lane l accumulates components x,y,z,w of elements 4l..4l+3 of each
// 128-float segment in four FMA chains, combines them as (x+y)+(z+w), and a
// butterfly sum across the warp finishes (every lane returns the same bits).
// p and r: 16-byte aligned, ldN a multiple of 4, zero padded past N.
MP_DEV float dot1(const float* __restrict__ p, const float* __restrict__ r, int ldN, int lane) {
    float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
#pragma unroll 4
    for (int off = lane * 4; off < ldN; off += 128) {
        const float4 q = *reinterpret_cast<const float4*>(r + off);
        const float4 v = *reinterpret_cast<const float4*>(p + off);
        ax = fmaf(v.x, q.x, ax);
        ay = fmaf(v.y, q.y, ay);
        az = fmaf(v.z, q.z, az);
        aw = fmaf(v.w, q.w, aw);
    }
    return warp_sum_f32((ax + ay) + (az + aw));
}

// Four consecutive atoms (stride ldN) at once, same order per atom as dot1.
MP_DEV void dot4(const float* __restrict__ p, const float* __restrict__ r, int ldN, int lane, float out[4]) {
    float a[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i][0] = a[i][1] = a[i][2] = a[i][3] = 0.f;
#pragma unroll 2
    for (int off = lane * 4; off < ldN; off += 128) {
        const float4 q = *reinterpret_cast<const float4*>(r + off);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 v = *reinterpret_cast<const float4*>(p + static_cast<size_t>(i) * ldN + off);
            a[i][0] = fmaf(v.x, q.x, a[i][0]);
            a[i][1] = fmaf(v.y, q.y, a[i][1]);
            a[i][2] = fmaf(v.z, q.z, a[i][2]);
            a[i][3] = fmaf(v.w, q.w, a[i][3]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = warp_sum_f32((a[i][0] + a[i][1]) + (a[i][2] + a[i][3]));
}

}  // namespace mpgb

namespace mpgb {

// FP64 correlation with its own fixed order.  The 64-double segments of
// the row fall in 4 classes (segment index mod 4); lane l accumulates
// elements 2l, 2l+1 of the segments of class q in two FMA chains x_q, y_q
// (increasing segment index), forms p_q = x_q + y_q, combines
// (p_0 + p_1) + (p_2 + p_3), and a butterfly sum across the warp finishes.
// The class split lets four warps share one atom (warp q computing p_q)
// with the same bits as one warp computing all four.  p and r 16-byte
// aligned, ldN a multiple of 2, zero padded past N.
MP_DEV double dot1(const double* __restrict__ p, const double* __restrict__ r, int ldN, int lane) {
    double ax[4] = {0.0, 0.0, 0.0, 0.0}, ay[4] = {0.0, 0.0, 0.0, 0.0};
    for (int base = lane * 2; base < ldN; base += 256) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int off = base + 64 * q;
            if (off < ldN) {
                const double2 u = *reinterpret_cast<const double2*>(r + off);
                const double2 v = *reinterpret_cast<const double2*>(p + off);
                ax[q] = fma(v.x, u.x, ax[q]);
                ay[q] = fma(v.y, u.y, ay[q]);
            }
        }
    }
    return warp_sum_f64(((ax[0] + ay[0]) + (ax[1] + ay[1])) + ((ax[2] + ay[2]) + (ax[3] + ay[3])));
}

// Four consecutive FP64 atoms (stride ldN), same order per atom as dot1.
MP_DEV void dot4(const double* __restrict__ p, const double* __restrict__ r, int ldN, int lane, double out[4]) {
    double ax[4][4], ay[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) ax[i][q] = ay[i][q] = 0.0;
    for (int base = lane * 2; base < ldN; base += 256) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int off = base + 64 * q;
            if (off < ldN) {
                const double2 u = *reinterpret_cast<const double2*>(r + off);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const double2 v = *reinterpret_cast<const double2*>(p + static_cast<size_t>(i) * ldN + off);
                    ax[i][q] = fma(v.x, u.x, ax[i][q]);
                    ay[i][q] = fma(v.y, u.y, ay[i][q]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
        out[i] = warp_sum_f64(((ax[i][0] + ay[i][0]) + (ax[i][1] + ay[i][1])) +
                              ((ax[i][2] + ay[i][2]) + (ax[i][3] + ay[i][3])));
}

}  // namespace mpgb
