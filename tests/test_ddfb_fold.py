"""The algebra the first DDFB dual layer relies on (Sec. II-B, Example 2),
checked on the CPU with the oracle's analysis operator and its adjoint:
W_1^* W_K v equals a 5 x 5 correlation of v with
C[e][f] = sum_p sum_{c - a = e - 2, d - b = f - 2} w_1[p][a][b] w_K[p][c][d]
wherever the nine pixels q - a + 1 lie inside the image, and everywhere equals
the sum over the inside (a, b) of sum_cd M[ab][cd] v(q - a + c, q - b + d) with
M[ab][cd] = sum_p w_1[p][ab] w_K[p][cd] (v zero outside the image)."""
import numpy as np

import synth


def test_first_layer_fold(orc):
    dd = synth.ddfb_weights(4, 16, 3)
    w1, wK = dd.filters[0], dd.filters[3]
    M = w1.reshape(16, 9).T @ wK.reshape(16, 9)
    C = np.zeros((5, 5))
    for ab in range(9):
        for cd in range(9):
            C[cd // 3 - ab // 3 + 2, cd % 3 - ab % 3 + 2] += M[ab, cd]
    rng = np.random.default_rng(1)
    ny, nx = 13, 17
    v = rng.random((ny, nx))
    ref = orc.ddfb_Wt(orc.ddfb_W(v, wK), w1)
    vp = np.pad(v, 2)
    for i in range(ny):
        for j in range(nx):
            folded = 0.0
            for a in range(3):
                for b in range(3):
                    if 0 <= i - a + 1 < ny and 0 <= j - b + 1 < nx:
                        for c in range(3):
                            for d in range(3):
                                folded += M[a * 3 + b, c * 3 + d] * vp[i - a + c + 2, j - b + d + 2]
            assert abs(folded - ref[i, j]) <= 1e-13
            if 1 <= i <= ny - 2 and 1 <= j <= nx - 2:
                assert abs((C * vp[i:i + 5, j:j + 5]).sum() - ref[i, j]) <= 1e-13
