// lattice.cuh -- velocity sets of the coupled LB-EHD step as compile-time traits.
//
// Flow / phase-field lattice: D2Q9 or D3Q19 with the weights printed after Eq. 16
// (3D: 1/3, 1/18, 1/36) and c_s^2 = 1/3. Charge lattice: D2Q5 (w0 = 1/3, c_s^2 = 1/3) or
// D3Q7 (w0 = 1/4, c_s^2 = 1/4). Velocity order: rest, then pairs (v, -v); the charge
// lattice is the first 2D+1 velocities of the flow lattice.
#pragma once

namespace lbehd {

template <int D>
struct Lat;

template <>
struct Lat<2> {
    static constexpr int Q = 9;
    static constexpr int QS = 5;
    static constexpr float cs2 = 1.0f / 3.0f;
    static constexpr float cs2s = 1.0f / 3.0f;
    __host__ __device__ static constexpr int ex(int n)
    {
        constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
        return t[n];
    }
    __host__ __device__ static constexpr int ey(int n)
    {
        constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        return t[n];
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr float w(int n)
    {
        return n == 0 ? 4.0f / 9.0f : (n < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
    }
    __host__ __device__ static constexpr float ws(int n) { return n == 0 ? 1.0f / 3.0f : 1.0f / 6.0f; }
};

template <>
struct Lat<3> {
    static constexpr int Q = 19;
    static constexpr int QS = 7;
    static constexpr float cs2 = 1.0f / 3.0f;
    static constexpr float cs2s = 1.0f / 4.0f;
    __host__ __device__ static constexpr int ex(int n)
    {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[n];
    }
    __host__ __device__ static constexpr int ey(int n)
    {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[n];
    }
    __host__ __device__ static constexpr int ez(int n)
    {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[n];
    }
    __host__ __device__ static constexpr float w(int n)
    {
        return n == 0 ? 1.0f / 3.0f : (n < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
    }
    __host__ __device__ static constexpr float ws(int n) { return n == 0 ? 0.25f : 0.125f; }
};

__host__ __device__ constexpr int opposite(int n) { return n == 0 ? 0 : ((n & 1) ? n + 1 : n - 1); }

}  // namespace lbehd
