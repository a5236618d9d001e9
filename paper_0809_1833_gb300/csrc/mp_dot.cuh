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

// FP64 correlation with its own fixed order: lane l accumulates elements
// 2l, 2l+1 of each 64-double segment in two FMA chains, adds them, and a
// butterfly sum across the warp finishes.  p and r 16-byte aligned, ldN a
// multiple of 2, zero padded past N.
MP_DEV double dot1(const double* __restrict__ p, const double* __restrict__ r, int ldN, int lane) {
    double ax = 0.0, ay = 0.0;
#pragma unroll 4
    for (int off = lane * 2; off < ldN; off += 64) {
        const double2 q = *reinterpret_cast<const double2*>(r + off);
        const double2 v = *reinterpret_cast<const double2*>(p + off);
        ax = fma(v.x, q.x, ax);
        ay = fma(v.y, q.y, ay);
    }
    return warp_sum_f64(ax + ay);
}

// Four consecutive FP64 atoms (stride ldN), same order per atom as dot1.
MP_DEV void dot4(const double* __restrict__ p, const double* __restrict__ r, int ldN, int lane, double out[4]) {
    double a[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i][0] = a[i][1] = 0.0;
#pragma unroll 2
    for (int off = lane * 2; off < ldN; off += 64) {
        const double2 q = *reinterpret_cast<const double2*>(r + off);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double2 v = *reinterpret_cast<const double2*>(p + static_cast<size_t>(i) * ldN + off);
            a[i][0] = fma(v.x, q.x, a[i][0]);
            a[i][1] = fma(v.y, q.y, a[i][1]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = warp_sum_f64(a[i][0] + a[i][1]);
}

}  // namespace mpgb
