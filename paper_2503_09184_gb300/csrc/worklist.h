// worklist.h -- device work list of the matmul kernels (filled on the host).
#pragma once
#include "rns.h"

struct MmDesc {
    const u32* A_ext;  // [nct_A][2][K][N] (tensor base B, NTT form)
    const u32* B_ext;  // [rows_B * Nc][2][K][N]
    u64* C;            // [M*Nc][2][L][N]
    int Nc;
    int group;  // products per scale-and-round: 1 (Alg. 1), or the grouped mode's size
};

struct Entry {
    int mm;     // matmul index
    int row;    // i
    int col;    // j
    int count;  // products
    int first;  // first (a_idx, k) pair in the row list
    int pad[3];
};
