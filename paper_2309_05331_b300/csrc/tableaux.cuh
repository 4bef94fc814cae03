// tableaux.cuh -- Butcher tableaux of the explicit Runge-Kutta steppers of
// Table 1 (explicit Euler, modified midpoint, RK4, Dormand-Prince 5(4),
// Cash-Karp 5(4), Fehlberg 7(8)) as compile-time constants for host and device code: the
// pointwise ensemble kernels (ode_tableau.cu) unroll them into FMA chains,
// and the Gray-Scott tableau path (gs_grid.cu) reads them on the host.
// Each struct: S stages, P / Q the orders of the propagated / embedded
// solutions (Q = 0: no embedded solution), c(i), a(i, j) (strictly lower
// triangular, row i = stage i+1), b(i) propagated weights, bh(i) embedded.
#pragma once

namespace gsk {

struct TabEuler {
    static constexpr int S = 1, P = 1, Q = 0;
    __host__ __device__ static constexpr double c(int i) {
        constexpr double v[1] = {0.0};
        return v[i];
    }
    __host__ __device__ static constexpr double a(int i, int j) {
        constexpr double v[1][1] = {{0.0}};
        return v[i][j];
    }
    __host__ __device__ static constexpr double b(int i) {
        constexpr double v[1] = {1.0};
        return v[i];
    }
    __host__ __device__ static constexpr double bh(int i) {
        constexpr double v[1] = {0.0};
        return v[i];
    }
};
// modified midpoint with two substeps (z1 = y + h f(y), z2 = y + 2h f(z1),
// y' = (z1 + z2 + h f(z2)) / 2, h = dt / 2) as a 3-stage tableau; order 2.
struct TabMidpoint {
    static constexpr int S = 3, P = 2, Q = 0;
    __host__ __device__ static constexpr double c(int i) {
        constexpr double v[3] = {0.0, 0.5, 1.0};
        return v[i];
    }
    __host__ __device__ static constexpr double a(int i, int j) {
        constexpr double v[3][3] = {{0, 0, 0}, {0.5, 0, 0}, {0, 1.0, 0}};
        return v[i][j];
    }
    __host__ __device__ static constexpr double b(int i) {
        constexpr double v[3] = {0.25, 0.5, 0.25};
        return v[i];
    }
    __host__ __device__ static constexpr double bh(int i) {
        constexpr double v[3] = {0.0, 0.0, 0.0};
        return v[i];
    }
};
struct TabRK4 {
    static constexpr int S = 4, P = 4, Q = 0;
    __host__ __device__ static constexpr double c(int i) {
        constexpr double v[4] = {0.0, 0.5, 0.5, 1.0};
        return v[i];
    }
    __host__ __device__ static constexpr double a(int i, int j) {
        constexpr double v[4][4] = {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1.0, 0}};
        return v[i][j];
    }
    __host__ __device__ static constexpr double b(int i) {
        constexpr double v[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
        return v[i];
    }
    __host__ __device__ static constexpr double bh(int i) {
        constexpr double v[4] = {0, 0, 0, 0};
        return v[i];
    }
};
struct TabDP5 {
    static constexpr int S = 7, P = 5, Q = 4;
    __host__ __device__ static constexpr double c(int i) {
        constexpr double v[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
        return v[i];
    }
    __host__ __device__ static constexpr double a(int i, int j) {
        constexpr double v[7][7] = {
        {0, 0, 0, 0, 0, 0, 0},
        {dp5::A21, 0, 0, 0, 0, 0, 0},
        {dp5::A31, dp5::A32, 0, 0, 0, 0, 0},
        {dp5::A41, dp5::A42, dp5::A43, 0, 0, 0, 0},
        {dp5::A51, dp5::A52, dp5::A53, dp5::A54, 0, 0, 0},
        {dp5::A61, dp5::A62, dp5::A63, dp5::A64, dp5::A65, 0, 0},
        {dp5::B1, 0, dp5::B3, dp5::B4, dp5::B5, dp5::B6, 0}};
        return v[i][j];
    }
    __host__ __device__ static constexpr double b(int i) {
        constexpr double v[7] = {dp5::B1, 0, dp5::B3, dp5::B4, dp5::B5, dp5::B6, 0};
        return v[i];
    }
    __host__ __device__ static constexpr double bh(int i) {
        constexpr double v[7] = {dp5::H1, 0, dp5::H3, dp5::H4, dp5::H5, dp5::H6, dp5::H7};
        return v[i];
    }
};
// Cash & Karp (1990): order-5 solution propagated, order-4 embedded.
struct TabCK54 {
    static constexpr int S = 6, P = 5, Q = 4;
    __host__ __device__ static constexpr double c(int i) {
        constexpr double v[6] = {0.0, 1.0 / 5, 3.0 / 10, 3.0 / 5, 1.0, 7.0 / 8};
        return v[i];
    }
    __host__ __device__ static constexpr double a(int i, int j) {
        constexpr double v[6][6] = {{0, 0, 0, 0, 0, 0},
                                       {1.0 / 5, 0, 0, 0, 0, 0},
                                       {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
                                       {3.0 / 10, -9.0 / 10, 6.0 / 5, 0, 0, 0},
                                       {-11.0 / 54, 5.0 / 2, -70.0 / 27, 35.0 / 27, 0, 0},
                                       {1631.0 / 55296, 175.0 / 512, 575.0 / 13824, 44275.0 / 110592,
                                        253.0 / 4096, 0}};
        return v[i][j];
    }
    __host__ __device__ static constexpr double b(int i) {
        constexpr double v[6] = {37.0 / 378, 0, 250.0 / 621, 125.0 / 594, 0, 512.0 / 1771};
        return v[i];
    }
    __host__ __device__ static constexpr double bh(int i) {
        constexpr double v[6] = {2825.0 / 27648, 0, 18575.0 / 48384, 13525.0 / 55296, 277.0 / 14336,
                                     1.0 / 4};
        return v[i];
    }
};
// Fehlberg (1968) 7(8), 13 stages; Table 1 lists it as order 8: the order-8
// weights are propagated, the order-7 ones embedded.
struct TabRKF78 {
    static constexpr int S = 13, P = 8, Q = 7;
    __host__ __device__ static constexpr double c(int i) {
        constexpr double v[13] = {0.0,       2.0 / 27, 1.0 / 9, 1.0 / 6, 5.0 / 12, 1.0 / 2, 5.0 / 6,
                                     1.0 / 6,   2.0 / 3,  1.0 / 3, 1.0,     0.0,      1.0};
        return v[i];
    }
    __host__ __device__ static constexpr double a(int i, int j) {
        constexpr double v[13][13] = {
        {0},
        {2.0 / 27},
        {1.0 / 36, 1.0 / 12},
        {1.0 / 24, 0, 1.0 / 8},
        {5.0 / 12, 0, -25.0 / 16, 25.0 / 16},
        {1.0 / 20, 0, 0, 1.0 / 4, 1.0 / 5},
        {-25.0 / 108, 0, 0, 125.0 / 108, -65.0 / 27, 125.0 / 54},
        {31.0 / 300, 0, 0, 0, 61.0 / 225, -2.0 / 9, 13.0 / 900},
        {2.0, 0, 0, -53.0 / 6, 704.0 / 45, -107.0 / 9, 67.0 / 90, 3.0},
        {-91.0 / 108, 0, 0, 23.0 / 108, -976.0 / 135, 311.0 / 54, -19.0 / 60, 17.0 / 6, -1.0 / 12},
        {2383.0 / 4100, 0, 0, -341.0 / 164, 4496.0 / 1025, -301.0 / 82, 2133.0 / 4100, 45.0 / 82, 45.0 / 164,
         18.0 / 41},
        {3.0 / 205, 0, 0, 0, 0, -6.0 / 41, -3.0 / 205, -3.0 / 41, 3.0 / 41, 6.0 / 41},
        {-1777.0 / 4100, 0, 0, -341.0 / 164, 4496.0 / 1025, -289.0 / 82, 2193.0 / 4100, 51.0 / 82, 33.0 / 164,
         12.0 / 41, 0, 1.0}};
        return v[i][j];
    }
    __host__ __device__ static constexpr double b(int i) {
        constexpr double v[13] = {0, 0, 0, 0, 0, 34.0 / 105, 9.0 / 35, 9.0 / 35, 9.0 / 280, 9.0 / 280, 0,
                                     41.0 / 840, 41.0 / 840};
        return v[i];
    }
    __host__ __device__ static constexpr double bh(int i) {
        constexpr double v[13] = {41.0 / 840, 0, 0, 0, 0, 34.0 / 105, 9.0 / 35, 9.0 / 35, 9.0 / 280,
                                      9.0 / 280, 41.0 / 840, 0, 0};
        return v[i];
    }
};

}  // namespace gsk
