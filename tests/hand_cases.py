"""Hand-worked one-pixel GlassNet cases with widths shrunk to 2.

Widths: scene 2, latent Z = 2, transparency channels 2, G-buffer channels 2,
hidden H = 2, output 3.  Weights are small integers chosen so that every
weight block, every bias, both concat orders and both halves of the pool reach
the output with distinct values.  Each step below was worked by hand; the
expected logits are exact integers, so the expected RGB is the logistic
function of an integer (checked against scipy's ``expit``).
"""
import numpy as np

W = {
    # F1: [[1, 1], [0, -1]] s + [0, 3]; s = [1, 2] -> [3, 1] -> ReLU [3, 1]
    "F1": (np.array([[1, 1], [0, -1]], np.float32), np.array([0, 3], np.float32)),
    # F2: [[1, -1], [0, 2]] [3, 1] + [0, -1] -> [2, 1] -> sigma = [2, 1]
    "F2": (np.array([[1, -1], [0, 2]], np.float32), np.array([0, -1], np.float32)),
    # phi1 on [t0, t1, z0, z1]:
    #   t = [1, 0]: [1 + 2, 0 - 1 + 2] = [3, 1]
    #   t = [0, 1]: [0 + 2, 1 - 1 + 2] = [2, 2]
    "phi1": (np.array([[1, 0, 1, 0], [0, 1, 0, -1]], np.float32), np.array([0, 2], np.float32)),
    # phi2: [[1, 1], [-1, 2]] u + [1, 0]
    #   u = [3, 1]: [5, -1] -> v = [5, 0]   (ReLU clips)
    #   u = [2, 2]: [5, 2]  -> v = [5, 2]
    "phi2": (np.array([[1, 1], [-1, 2]], np.float32), np.array([1, 0], np.float32)),
    # rho on [max0, max1, mean0, mean1] with bias [0, 1]:
    #   one layer  t=[1,0]:        pool [5, 0, 5, 0] -> [5 - 0, 0 + 5 + 1] = [5, 6]
    #   two layers t=[1,0],[0,1]:  max [5, 2], mean [5, 1]
    #                              pool [5, 2, 5, 1] -> [5 - 1, 2 + 5 + 1] = [4, 8]
    "rho": (np.array([[1, 0, 0, -1], [0, 1, 1, 0]], np.float32), np.array([0, 1], np.float32)),
    # B1 on [g0, g1, r0, r1, z0, z1], g = [1, -1], bias [0, 1]:
    #   row 0 = g0 + r0 + z1, row 1 = 2 g1 + r1 + z0 + 1
    #   one layer  r = [5, 6]: [1 + 5 + 1, -2 + 6 + 2 + 1] = [7, 7]
    #   two layers r = [4, 8]: [1 + 4 + 1, -2 + 8 + 2 + 1] = [6, 9]
    #   no layer   r = [0, 0]: [1 + 0 + 1, -2 + 0 + 2 + 1] = [2, 1]
    "B1": (np.array([[1, 0, 1, 0, 0, 1], [0, 2, 0, 1, 1, 0]], np.float32),
           np.array([0, 1], np.float32)),
    # B2: [[2, -1], [1, 0]] y + [0, -1]
    #   [7, 7] -> [7, 6];  [6, 9] -> [3, 5];  [2, 1] -> [3, 1]
    "B2": (np.array([[2, -1], [1, 0]], np.float32), np.array([0, -1], np.float32)),
    # R1: [[1, 0], [-1, 1]] y + [0, 3]
    #   [7, 6] -> [7, 2];  [3, 5] -> [3, 5];  [3, 1] -> [3, 1]
    "R1": (np.array([[1, 0], [-1, 1]], np.float32), np.array([0, 3], np.float32)),
    # R2: [[1, -1], [0, 1], [-1, 0]] q + [0, 0, 1]
    #   [7, 2] -> [5, 2, -6];  [3, 5] -> [-2, 5, -2];  [3, 1] -> [2, 1, -2]
    "R2": (np.array([[1, -1], [0, 1], [-1, 0]], np.float32), np.array([0, 0, 1], np.float32)),
}

SCENE = np.array([1, 2], np.float32)
SIGMA = np.array([2.0, 1.0])
G = np.array([1, -1], np.float32)
LAYER_A = np.array([1, 0], np.float32)
LAYER_B = np.array([0, 1], np.float32)

# Expected pre-sigmoid outputs (exact integers) for each case.
LOGITS_ONE_LAYER = np.array([5.0, 2.0, -6.0])
LOGITS_TWO_LAYERS = np.array([-2.0, 5.0, -2.0])
LOGITS_NO_LAYER = np.array([2.0, 1.0, -2.0])
POOL_TWO_LAYERS = np.array([5.0, 2.0, 5.0, 1.0])

# Sum pooling (the paper's Eq. 5 form, tau = sum_k v_k straight into B, no rho):
#   one layer  tau = [5, 0]:  B1 [1 + 5 + 1, 0 + 1] = [7, 1];  B2 [14 - 1, 7 - 1] = [13, 6]
#              R1 [13, -13 + 6 + 3] -> [13, 0];  R2 [13, 0, -13 + 1]
#   two layers tau = [10, 2]: B1 [12, 3];  B2 [24 - 3, 12 - 1] = [21, 11]
#              R1 [21, -21 + 11 + 3] -> [21, 0];  R2 [21, 0, -21 + 1]
#   no layer   tau = [0, 0]:  the opaque-only logits above
TAU_TWO_LAYERS = np.array([10.0, 2.0])
LOGITS_SUM_ONE_LAYER = np.array([13.0, 0.0, -12.0])
LOGITS_SUM_TWO_LAYERS = np.array([21.0, 0.0, -20.0])

# Positional encoding with L = 1: every input x of n channels enters as
# [x ; sin(pi x) ; cos(pi x)] (3n columns, blocks in that order).  Inputs are
# multiples of 1/2, so every sine and cosine is 0 or +-1 (to within 2^-52).
#   scene s = [1/2, 1]  -> [0.5, 1, 1, 0, 0, -1]
#   F1 rows [2, 0, 1, 0, 0, 0] and [0, 1, 0, 0, 0, -1], bias [0, 1]:
#     [1 + 1, 1 + 1 + 1] = [2, 3];  F2 [[1, -1], [0, 1]] + [2, -1]: sigma = [1, 2]
#   layer A = [1/2, 0]  -> [0.5, 0, 1, 0, 0, 1]
#   layer B = [1, 1/2]  -> [1, 0.5, 0, 1, -1, 0]
#   phi1 on [gamma(t) ; z0 ; z1], rows [2, 0, 3, 0, 0, 0, 1, 0], [0, 2, 0, 1, 0, -1, 0, 1]:
#     A: [1 + 3 + 1, -1 + 2] = [5, 1];  B: [2 + 0 + 1, 1 + 1 + 2] = [3, 4]
#   phi2 (as W): A [5 + 1 + 1, -5 + 2] -> v_A = [7, 0];  B [3 + 4 + 1, -3 + 8] -> v_B = [8, 5]
#   rho (as W): one layer pool [7, 0, 7, 0] -> [7, 8]
#               two layers max [8, 5], mean [7.5, 2.5] -> [8 - 2.5, 5 + 7.5 + 1] = [5.5, 13.5]
#   g = [1/2, -1] -> [0.5, -1, 1, 0, 0, -1]
#   B1 on [gamma(g) ; r ; z], rows [2, 0, 1, 0, 0, 0, 1, 0, 0, 1], [0, 1, 0, 0, 0, -2, 0, 1, 1, 0]:
#     row 0 = 1 + 1 + r0 + 2 = 4 + r0, row 1 = -1 + 2 + r1 + 1 = 2 + r1
#     one layer [11, 10];  two layers [9.5, 15.5];  no layer [4, 2]
#   B2 [[1, -1], [0, 1]]: [1, 10];  [-6 -> 0, 15.5];  [2, 2]
#   R1 [[1, 0], [-1, 1]] + [0, 1]: [1, 10];  [0, 16.5];  [2, 1]
#   R2 (as W): [-9, 10, 0];  [-16.5, 16.5, 1];  [1, 1, -1]
#   sum pooling: tau one layer [7, 0] -> B1 [11, 2] -> B2 [9, 2] -> R1 [9, 0] -> R2 [9, 0, -8]
#                tau two layers [15, 5] -> B1 [19, 7] -> B2 [12, 7] -> R1 [12, 0] -> R2 [12, 0, -11]
W_PE = dict(W)
W_PE.update({
    "F1": (np.array([[2, 0, 1, 0, 0, 0], [0, 1, 0, 0, 0, -1]], np.float32), np.array([0, 1], np.float32)),
    "F2": (np.array([[1, -1], [0, 1]], np.float32), np.array([2, -1], np.float32)),
    "phi1": (np.array([[2, 0, 3, 0, 0, 0, 1, 0], [0, 2, 0, 1, 0, -1, 0, 1]], np.float32),
             np.array([0, 0], np.float32)),
    "B1": (np.array([[2, 0, 1, 0, 0, 0, 1, 0, 0, 1], [0, 1, 0, 0, 0, -2, 0, 1, 1, 0]], np.float32),
           np.array([0, 0], np.float32)),
    "B2": (np.array([[1, -1], [0, 1]], np.float32), np.array([0, 0], np.float32)),
    "R1": (np.array([[1, 0], [-1, 1]], np.float32), np.array([0, 1], np.float32)),
    "pe_freqs": 1,
})
SCENE_PE = np.array([0.5, 1.0], np.float32)
SIGMA_PE = np.array([1.0, 2.0])
G_PE = np.array([0.5, -1.0], np.float32)
LAYER_PA = np.array([0.5, 0.0], np.float32)
LAYER_PB = np.array([1.0, 0.5], np.float32)
LOGITS_PE_ONE_LAYER = np.array([-9.0, 10.0, 0.0])
LOGITS_PE_TWO_LAYERS = np.array([-16.5, 16.5, 1.0])
LOGITS_PE_NO_LAYER = np.array([1.0, 1.0, -1.0])
LOGITS_PE_SUM_ONE_LAYER = np.array([9.0, 0.0, -8.0])
LOGITS_PE_SUM_TWO_LAYERS = np.array([12.0, 0.0, -11.0])

# Spatial R: R1 as a 3x3 kernel over the neural buffer y (B's output) of a
# 2x2 frame, the network W otherwise.  Pixels: (0,0) layer A -> y = [7, 6];
# (0,1) layers A, B -> [3, 5]; (1,0) no layer -> [3, 1]; (1,1) B, A -> [3, 5].
# Kernel [out][in][ky][kx] (tap (dy, dx) at [dy + 1][dx + 1]):
#   out 0 = in 0 at the centre + in 1 of the right neighbour
#   out 1 = in 0 of the neighbour below - in 1 at the centre, bias 3
#   (0,0): [7 + 5, 3 - 6 + 3] = [12, 0]     (0,1): [3 + 0, 3 - 5 + 3] = [3, 1]
#   (1,0): [3 + 5, 0 - 1 + 3] = [8, 2]      (1,1): [3 + 0, 0 - 5 + 3] -> [3, 0]
#   R2 (as W): [12, 0, -11];  [2, 1, -2];  [6, 2, -7];  [3, 0, -2]
_K3 = np.zeros((2, 2, 3, 3), np.float32)
_K3[0, 0, 1, 1] = 1
_K3[0, 1, 1, 2] = 1
_K3[1, 0, 2, 1] = 1
_K3[1, 1, 1, 1] = -1
W_R3 = dict(W)
W_R3["R1"] = (_K3.reshape(2, 18), np.array([0, 3], np.float32))
W_R3["r_kernel"] = 3
LOGITS_R3 = np.array([[[12.0, 2.0], [6.0, 3.0]],
                      [[0.0, 1.0], [2.0, 0.0]],
                      [[-11.0, -2.0], [-7.0, -2.0]]])  # [3][h][w]
