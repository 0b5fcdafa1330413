// Compiled (D, P) variants of the DP kernel.  P is the number of band cells
// a lane computes per anti-diagonal; the ring buffers hold 2*(P+1)*D floats,
// so P shrinks as D grows to stay within the register file.
#pragma once

#define KNN_DP_VARIANTS(X)                                                         \
    X(1, 2) X(1, 4) X(1, 7) X(1, 13)                                               \
    X(2, 2) X(2, 4) X(2, 7) X(2, 13)                                               \
    X(3, 2) X(3, 4) X(3, 7) X(3, 13)                                               \
    X(4, 2) X(4, 4) X(4, 7)                                                        \
    X(5, 2) X(5, 4) X(5, 7)                                                        \
    X(6, 2) X(6, 4) X(6, 7)                                                        \
    X(7, 2) X(7, 4)                                                                \
    X(8, 2) X(8, 4)                                                                \
    X(16, 2) X(16, 4)
