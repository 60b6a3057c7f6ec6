"""Algorithmic work of the MPPI hot path, for the roofline.

FLOPs are counted per structured operation of the algorithm as formulated in
the kernels (FMA = 2, add/sub/mul = 1, divide/sqrt = 1; sin/cos are listed
separately and not counted), once per rollout: work a kernel replicates across
lanes (the trunk solve runs on all 4 lanes of a rollout) counts once, and
symmetric 3x3 blocks count their 6 unique entries.  Bytes are the unique
global-memory bytes an ideal kernel moves.
"""

# ---- per structured op
ROT3_VEC = 6          # coordinate rotation of a 3-vector about x or y
CROSS = 9
ADD3 = 3
SYM6_MV = 72          # dense 6x6 times 6-vector
BIAS = SYM6_MV + 3 * CROSS + 2 * ADD3 + 6          # v x* I v - f_ext
PROJECT = (6 + 21 * 2) + (SYM6_MV + 1 + 12 + 6)     # Ia = IA - U U^T/D ; pa = pA + Ia c + U u/D
UDU = 3                                            # D = U_k + a, 1/D, u = tau - pA_k
FORCE_XFORM = 2 * ROT3_VEC + CROSS + ADD3          # X^T f
CONGRUENCE = (30 + 36 + 30) + (27 + 27 + 18 + 18 + 9)   # rotate blocks; translate (P, T, Q, A'', B'')
ADD_I = 21
KIN_BODY = ROT3_VEC + (CROSS + ADD3) + ROT3_VEC + 1 + 4   # v = X v_p + S qd ; c = v x S qd
PASS3_BODY = 24 + 6 + 11 + 2 + 1
PD_JOINT = 6
INT_JOINT = 4
FOOT_FK = 3 * (ROT3_VEC + ADD3) + 15 + 3
NORMAL_TO_BODY = 15 + 3 * ROT3_VEC
GROUND_PLANE = 7
CONTACT = 65

LEG = (3 * KIN_BODY + 3 * PD_JOINT
       + (BIAS + UDU + PROJECT + FORCE_XFORM + CONGRUENCE)            # calf
       + 2 * (ADD_I + BIAS + UDU + PROJECT + FORCE_XFORM + CONGRUENCE)  # thigh, hip
       + 3 * PASS3_BODY + 3 * INT_JOINT
       + FOOT_FK + NORMAL_TO_BODY + GROUND_PLANE + CONTACT)
TRUNK_SPHERE = 15 + 3 + 15 + GROUND_PLANE + 10     # typical: out of contact
TRUNK = (24                    # R from the quaternion
         + 27 * 3 + 6 * 3 + 6  # sum of the 4 legs' (IA, pA) and sphere wrenches
         + 30                  # the trunk's own bias and inertia
         + 82 + 72             # 6x6 Cholesky and two triangular solves
         + 90                  # semi-implicit Euler of the free base incl. quaternion
         + 3 * TRUNK_SPHERE)
SUBSTEP = 4 * LEG + TRUNK      # one rollout advanced by one sub-step
PER_DT_STEP = 4 * 22 + 12 * 3 * 2 + 60   # spline basis + targets + stage cost


def rollout_flops(K: int, H: int, n_sub: int) -> float:
    """Algorithmic FLOPs of one rollout-kernel launch over K samples."""
    return float(K) * H * (n_sub * SUBSTEP + PER_DT_STEP)


def sample_bytes(K: int) -> float:
    """K1: writes U[K][48] floats (reads 48 floats of mu)."""
    return 4.0 * K * 48 + 4 * 48


def update_bytes(K: int) -> float:
    """K3/K4: reads L[K] and U[K][48]; writes mu, u0."""
    return 4.0 * K * 49 + 4 * (48 + 48 + 12)


def fp32_peak_tflops(sms: int = 152, mhz: float = 2070.0) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12
