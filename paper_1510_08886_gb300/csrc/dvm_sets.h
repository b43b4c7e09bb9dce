// Generated by paper_1510_08886_gb300/gen_dvm_sets.py from the paper's DVM
// tables (App. A, App. B): compile-time +-e pair representatives of the
// velocity sets with register-resident specialised kernels.  Do not edit.
#pragma once

namespace lbm {

// S^{D2V16}_{Q7E58}: V = 16
struct SetD2V16 {
    static constexpr int R = 0, P = 8;
    static constexpr int ex[P] = {0, 1, 0, 2, 2, -2, 0, 4};
    static constexpr int ey[P] = {1, 0, 2, 0, 2, 2, 4, 0};
};

// S^{D2V32}_{Q7E944}: V = 32
struct SetD2V32 {
    static constexpr int R = 0, P = 16;
    static constexpr int ex[P] = {1, -1, 2, -2, 1, -1, 5, -5, 4, -4, 6, -6, 3, -3, 12, -12};
    static constexpr int ey[P] = {1, 1, 2, 2, 5, 5, 1, 1, 6, 6, 4, 4, 12, 12, 3, 3};
};

// S^{D2V33}_{Q9E132}: V = 33
struct SetD2V33 {
    static constexpr int R = 1, P = 16;
    static constexpr int ex[P] = {0, 1, 1, -1, 0, 2, 1, -1, 2, -2, 2, -2, 0, 3, 4, -4};
    static constexpr int ey[P] = {1, 0, 1, 1, 2, 0, 2, 2, 1, 1, 2, 2, 3, 0, 4, 4};
};

// (x, z) marginal of S^{D3V107}_{Q7E1023}: V = 53
struct SetD2V53 {
    static constexpr int R = 1, P = 26;
    static constexpr int ex[P] = {0, 1, 1, -1, 0, 2, 1, -1, 2, -2, 2, -2, 0, 3, 1, -1, 3, -3, 3, -3, 0, 5, 2, -2, 6, -6};
    static constexpr int ey[P] = {1, 0, 1, 1, 2, 0, 2, 2, 1, 1, 2, 2, 3, 0, 3, 3, 1, 1, 3, 3, 5, 0, 6, 6, 2, 2};
};

// (x, z) marginal of S^{D3V96}_{Q7E1932}: V = 40
struct SetD2V40 {
    static constexpr int R = 0, P = 20;
    static constexpr int ex[P] = {1, -1, 1, -1, 3, -3, 3, -3, 4, -4, 1, -1, 6, -6, 1, -1, 7, -7, 6, -6};
    static constexpr int ey[P] = {1, 1, 3, 3, 1, 1, 3, 3, 4, 4, 6, 6, 1, 1, 7, 7, 1, 1, 6, 6};
};

// (x, z) marginal of S^{D3V112}_{Q7E1764}: V = 48
struct SetD2V48 {
    static constexpr int R = 0, P = 24;
    static constexpr int ex[P] = {1, -1, 2, -2, 1, -1, 3, -3, 2, -2, 3, -3, 1, -1, 5, -5, 4, -4, 1, -1, 5, -5, 7, -7};
    static constexpr int ey[P] = {1, 1, 2, 2, 3, 3, 1, 1, 3, 3, 2, 2, 5, 5, 1, 1, 4, 4, 7, 7, 5, 5, 1, 1};
};

}  // namespace lbm
