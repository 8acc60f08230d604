// Generated by paper_2603_09038_gb300/smem_layout.py (do not edit): shared-memory strides of the
// fused apply kernel that minimise bank conflicts in a model of its warp accesses, keeping the
// elements per block of the default layout.  Key: D, Q, diffusion, element bytes, z re-read.
#pragma once

namespace fe {

struct SmemLayoutEntry {
  int D, Q, diff, es, rr;
  int s_dd, s_qd, s_qq, sz_a, sz_b;
};

constexpr SmemLayoutEntry kSmemLayouts[] = {
    {2, 3, 0, 4, 1, 6, 8, 9, 41, 38},  // NE 64: 920 -> 684 wavefronts
    {2, 3, 0, 8, 0, 5, 7, 9, 28, 22},  // NE 64: 1504 -> 1184 wavefronts
    {2, 3, 0, 8, 1, 4, 7, 11, 25, 22},  // NE 64: 1888 -> 1384 wavefronts
    {2, 3, 1, 4, 1, 6, 6, 9, 55, 70},  // NE 64: 3152 -> 1980 wavefronts
    {2, 3, 1, 8, 0, 5, 8, 9, 60, 86},  // NE 64: 4112 -> 2656 wavefronts
    {2, 3, 1, 8, 1, 4, 7, 11, 73, 70},  // NE 64: 4976 -> 3144 wavefronts
    {3, 4, 0, 4, 1, 12, 12, 16, 48, 59},  // NE 64: 2748 -> 2450 wavefronts
    {3, 4, 0, 8, 0, 10, 12, 18, 57, 49},  // NE 64: 4632 -> 3512 wavefronts
    {3, 4, 0, 8, 1, 10, 12, 18, 57, 49},  // NE 64: 5208 -> 4088 wavefronts
    {3, 4, 1, 4, 1, 12, 13, 18, 176, 172},  // NE 32: 3504 -> 2483 wavefronts
    {3, 4, 1, 8, 0, 10, 13, 18, 169, 156},  // NE 32: 3702 -> 3384 wavefronts
    {3, 4, 1, 8, 1, 10, 13, 18, 169, 156},  // NE 32: 4566 -> 4248 wavefronts
    {4, 5, 0, 4, 1, 18, 20, 25, 112, 107},  // NE 32: 3240 -> 2840 wavefronts
    {4, 5, 0, 8, 0, 19, 20, 26, 105, 100},  // NE 32: 4312 -> 3216 wavefronts
    {4, 5, 0, 8, 1, 19, 20, 26, 105, 100},  // NE 32: 5592 -> 4016 wavefronts
    {4, 5, 1, 4, 1, 17, 24, 26, 313, 372},  // NE 16: 4064 -> 2620 wavefronts
    {4, 5, 1, 8, 0, 19, 20, 26, 313, 308},  // NE 16: 4816 -> 3448 wavefronts
    {4, 5, 1, 8, 1, 19, 20, 26, 313, 308},  // NE 16: 6736 -> 4648 wavefronts
    {5, 6, 0, 4, 1, 28, 30, 36, 185, 190},  // NE 32: 5891 -> 5215 wavefronts
    {5, 6, 0, 8, 1, 25, 30, 36, 180, 190},  // NE 32: 9442 -> 8628 wavefronts
    {5, 6, 1, 4, 1, 28, 30, 38, 580, 542},  // NE 8: 3954 -> 2853 wavefronts
    {5, 6, 1, 8, 1, 25, 30, 38, 580, 542},  // NE 8: 5652 -> 4830 wavefronts
    {6, 7, 0, 4, 1, 37, 42, 50, 305, 298},  // NE 16: 4903 -> 3894 wavefronts
    {6, 7, 0, 8, 1, 39, 42, 49, 305, 295},  // NE 16: 8478 -> 7414 wavefronts
    {6, 7, 1, 4, 1, 37, 42, 50, 913, 906},  // NE 4: 3040 -> 2367 wavefronts
    {6, 7, 1, 8, 1, 39, 42, 49, 897, 890},  // NE 4: 5133 -> 4367 wavefronts
    {7, 8, 0, 4, 1, 52, 57, 64, 465, 472},  // NE 8: 3353 -> 2912 wavefronts
    {7, 8, 0, 8, 1, 50, 57, 64, 449, 456},  // NE 8: 5835 -> 5626 wavefronts
    {7, 8, 1, 4, 1, 52, 57, 67, 1407, 1368},  // NE 4: 3735 -> 3512 wavefronts
    {7, 8, 1, 8, 1, 50, 57, 64, 1345, 1368},  // NE 4: 7006 -> 6763 wavefronts
    {8, 9, 0, 4, 1, 67, 72, 83, 689, 648},  // NE 8: 5980 -> 4760 wavefronts
    {8, 9, 0, 8, 1, 65, 72, 81, 657, 648},  // NE 8: 10016 -> 9440 wavefronts
    {8, 9, 1, 4, 1, 67, 72, 83, 2001, 1960},  // NE 2: 3426 -> 2865 wavefronts
    {8, 9, 1, 8, 1, 65, 73, 81, 1953, 1976},  // NE 2: 5634 -> 5348 wavefronts
    {9, 10, 0, 4, 1, 81, 90, 103, 932, 922},  // NE 4: 3658 -> 3293 wavefronts
    {9, 10, 0, 8, 1, 81, 90, 101, 916, 906},  // NE 4: 6291 -> 5718 wavefronts
    {9, 10, 1, 4, 1, 81, 90, 102, 2756, 2714},  // NE 2: 4456 -> 4088 wavefronts
    {9, 10, 1, 8, 1, 81, 90, 101, 2740, 2714},  // NE 2: 7777 -> 7230 wavefronts
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};

}  // namespace fe
