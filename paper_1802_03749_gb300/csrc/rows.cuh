// Loads of a cell's or node's values from global memory and rows of values
// in shared memory, shared by the staged flux kernels (res_calc and its
// adjoint).
#pragma once

#include "common.cuh"

// q of cell g (4 values), AoS (one or two vector loads) or SoA
template <typename T, bool SOA>
__device__ __forceinline__ void load_cell(const T *__restrict__ q, int64_t ncell, int g, T &r, T &ru, T &rv, T &E)
{
    if (SOA) {
        r = q[g];
        ru = q[ncell + g];
        rv = q[2 * ncell + g];
        E = q[3 * ncell + g];
    } else if (sizeof(T) == 8) {
        const double2 *q2 = reinterpret_cast<const double2 *>(q) + 2 * (int64_t)g;
        double2 a = q2[0], b = q2[1];
        r = (T)a.x;
        ru = (T)a.y;
        rv = (T)b.x;
        E = (T)b.y;
    } else {
        float4 a = reinterpret_cast<const float4 *>(q)[g];
        r = (T)a.x;
        ru = (T)a.y;
        rv = (T)a.z;
        E = (T)a.w;
    }
}

// x of node g (2 values), AoS (one vector load) or SoA
template <typename T, bool SOA>
__device__ __forceinline__ void load_node(const T *__restrict__ x, int64_t nnode, int g, T &px, T &py)
{
    if (SOA) {
        px = x[g];
        py = x[nnode + g];
    } else if (sizeof(T) == 8) {
        double2 a = reinterpret_cast<const double2 *>(x)[g];
        px = (T)a.x;
        py = (T)a.y;
    } else {
        float2 a = reinterpret_cast<const float2 *>(x)[g];
        px = (T)a.x;
        py = (T)a.y;
    }
}

// Rows of 4 values in shared memory, one vector access each (16-byte
// aligned: float4, or two double2).
template <typename T>
__device__ __forceinline__ void st_row4(T *base, int i, T a, T b, T c, T d)
{
    if (sizeof(T) == 8) {
        double2 *p = reinterpret_cast<double2 *>(base) + 2 * i;
        p[0] = make_double2((double)a, (double)b);
        p[1] = make_double2((double)c, (double)d);
    } else {
        reinterpret_cast<float4 *>(base)[i] = make_float4((float)a, (float)b, (float)c, (float)d);
    }
}
template <typename T>
__device__ __forceinline__ void ld_row4(const T *base, int i, T &a, T &b, T &c, T &d)
{
    if (sizeof(T) == 8) {
        const double2 *p = reinterpret_cast<const double2 *>(base) + 2 * i;
        const double2 u = p[0], w = p[1];
        a = (T)u.x;
        b = (T)u.y;
        c = (T)w.x;
        d = (T)w.y;
    } else {
        const float4 u = reinterpret_cast<const float4 *>(base)[i];
        a = (T)u.x;
        b = (T)u.y;
        c = (T)u.z;
        d = (T)u.w;
    }
}

// -v by flipping the sign bit: an integer operation, so FP64 negations
// do not occupy the FP64 pipe
__device__ __forceinline__ float flip_sign(float v) { return __int_as_float(__float_as_int(v) ^ (int)0x80000000); }
__device__ __forceinline__ double flip_sign(double v)
{
    return __hiloint2double(__double2hiint(v) ^ (int)0x80000000, __double2loint(v));
}

// Rows of 2 values in shared memory (16 bytes: double2, or float2)
template <typename T>
__device__ __forceinline__ void st_row2(T *base, int i, T a, T b)
{
    if (sizeof(T) == 8)
        reinterpret_cast<double2 *>(base)[i] = make_double2((double)a, (double)b);
    else
        reinterpret_cast<float2 *>(base)[i] = make_float2((float)a, (float)b);
}
template <typename T>
__device__ __forceinline__ void ld_row2(const T *base, int i, T &a, T &b)
{
    if (sizeof(T) == 8) {
        const double2 u = reinterpret_cast<const double2 *>(base)[i];
        a = (T)u.x;
        b = (T)u.y;
    } else {
        const float2 u = reinterpret_cast<const float2 *>(base)[i];
        a = (T)u.x;
        b = (T)u.y;
    }
}

// Stores of a cell's 4 values / a node's 2 values to global memory, AoS
// (vector stores) or SoA
template <typename T, bool SOA>
__device__ __forceinline__ void store_cell(T *__restrict__ a, int64_t ncell, int64_t g, T v0, T v1, T v2, T v3)
{
    if (SOA) {
        a[g] = v0;
        a[ncell + g] = v1;
        a[2 * ncell + g] = v2;
        a[3 * ncell + g] = v3;
    } else if (sizeof(T) == 8) {
        double2 *p = reinterpret_cast<double2 *>(a) + 2 * g;
        p[0] = make_double2((double)v0, (double)v1);
        p[1] = make_double2((double)v2, (double)v3);
    } else {
        reinterpret_cast<float4 *>(a)[g] = make_float4((float)v0, (float)v1, (float)v2, (float)v3);
    }
}
template <typename T, bool SOA>
__device__ __forceinline__ void store_node(T *__restrict__ a, int64_t nnode, int64_t g, T v0, T v1)
{
    if (SOA) {
        a[g] = v0;
        a[nnode + g] = v1;
    } else if (sizeof(T) == 8) {
        reinterpret_cast<double2 *>(a)[g] = make_double2((double)v0, (double)v1);
    } else {
        reinterpret_cast<float2 *>(a)[g] = make_float2((float)v0, (float)v1);
    }
}
