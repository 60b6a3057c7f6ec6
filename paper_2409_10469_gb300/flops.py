"""Algorithmic work of the MPPI hot path, for the roofline.

FLOPs are counted per operation of the algorithm as formulated in the rollout
kernel (FMA = 2, add / sub / mul = 1, divide / sqrt / rsqrt = 1), once per
rollout: work a kernel replicates across the 4 lanes of a rollout (the trunk
solve) counts once, symmetric 3x3 blocks count their 6 unique entries, and
structurally-zero operands (joint offsets along one axis, centres of mass on
the joint axis, the plane's normal) count nothing.  Bytes are the unique
global-memory bytes an ideal kernel moves.
"""

# ---------------------------------------------------------------- one leg
SINCOS = 25                       # bounded sin/cos pair (reduction + 2 polynomials)
JOINT_SINCOS = 3 * SINCOS
KIN = 25 + 21 + 21                # body velocities + velocity products, hip/thigh/calf
FOOT_POS = 19 + 18                # foot in the trunk frame, then world
NORMAL_TO_CALF = 18               # plane normal into calf coordinates
GROUND_PLANE = 1
CONTACT = 64                      # spring-damper + regularised Coulomb + wrench
FOOT = FOOT_POS + NORMAL_TO_CALF + GROUND_PLANE + CONTACT
PD = 3 * 6
BIAS = 50                         # v x* I v - f_ext, structured body inertia
ROTATE_SYM6 = 20 + 36 + 20        # A, B, C blocks turned about one axis
CONG_KNEE = ROTATE_SYM6 + 33      # translation along z only
CONG_THIGH = ROTATE_SYM6 + 33     # translation along y only
CONG_HIP = ROTATE_SYM6 + 72       # translation in x and y
PROJECT = 6 + 24 + 18 + 48 + 1 + 12   # Ia = IA - U U^T / D ; pa = pA + Ia c + U u / D
FXFORM_1AX = 16                   # X^T f with a one-axis joint offset
FXFORM_HIP = 20
PASS2 = ((BIAS + 1 + 24 + FXFORM_1AX + CONG_KNEE)                       # calf (constant Ia)
         + (8 + BIAS + 6 + 3 + PROJECT + FXFORM_1AX + CONG_THIGH)        # thigh
         + (6 + 36 + 3 + PROJECT + FXFORM_HIP + CONG_HIP))               # hip
PASS3 = 40 + 34 + 25
INTEGRATE_LEG = 12
LEG = JOINT_SINCOS + KIN + FOOT + PD + PASS2 + PASS3 + INTEGRATE_LEG

# ---------------------------------------------------------------- trunk
TRUNK = (30          # rotation matrix of the quaternion
         + 99        # sums of the 4 legs' articulated inertias (21) and bias forces (6)
         + 30        # the trunk's own inertia and bias
         + 91 + 72   # 6x6 Cholesky and two triangular solves
         + 120       # semi-implicit Euler of the free base incl. quaternion
         + 3 * 7)    # trunk spheres against the plane (out of contact)

SUBSTEP_DYNAMICS = 4 * LEG + TRUNK  # one rollout advanced by one sub-step, plain FP32 geometry

# ---------------------------------------------------------------- precise contact geometry
# The per-step tolerance (1e-5 of the FP64 oracle per state block) needs the
# contact spheres' heights to ~1e-9 m, which plain FP32 misses by ~30x (the
# height is a difference of two ~0.3 m terms that k = 2e4 N/m amplifies).  The
# kernel therefore evaluates them as FP32 pairs (precise.cuh) from compensated
# angles, positions and attitude.  Counted like the rest, per operation of the
# formulation (TwoSum = 6 adds, Fast2Sum = 3, pair product = 1 mul + 4 FMA,
# pair x FP32 = 1 mul + 2 FMA, pair sum = TwoSum + 2 adds), as the difference
# to the plain formulation it replaces:
PAIR_SINCOS = 22                   # table point, exact reduction, third-order Taylor step, sin and cos
LEG_PRECISE = ((4 * PAIR_SINCOS + 8 + 6 - JOINT_SINCOS)   # q0, q1, q2, q1 + q2 as pairs; FP32 values
               + (154 - 37)                              # foot height as pairs, less the FP32 foot position
               + 6                                       # PD on the compensated angles
               + 3 * 7 - INTEGRATE_LEG)                  # joint updates with Fast2Sum compensation
TRUNK_PRECISE = (78                # row 2 of the attitude as pairs (exact products, lo corrections)
                 + 3 * (13 - 2)    # trunk-sphere heights as pairs
                 + 5               # attitude step as a compensated increment (no square root)
                 + 3)              # trunk height with Fast2Sum compensation
PRECISE = 4 * LEG_PRECISE + TRUNK_PRECISE
PER_DT_STEP_PRECISE = 49           # rounding the state at the dt step's end, the attitude's norm error

SUBSTEP = SUBSTEP_DYNAMICS + PRECISE   # the formulation the kernel runs (flat ground)

# The same sub-step as the FP64 oracle's plain formulation computes it (dense
# 6x6 spatial algebra, general rotations, no structural zeros dropped), counted
# operation by operation by the oracle's counting build (add/sub, mul, div, sqrt
# = 1; trot model, flat ground, from the stand state).  Context for SUBSTEP, which
# the roofline uses: the structured count is the smaller, conservative figure.
ORACLE_PLAIN_SUBSTEP = 23200
PER_DT_STEP = 112 + 180 + 25       # spline targets, per-leg control cost, trunk state cost


def rollout_flops(K: int, H: int, n_sub: int, precise: bool = True) -> float:
    """Algorithmic FLOPs of one rollout-kernel launch over K samples: the
    formulation the kernel runs (precise contact geometry included), or with
    precise=False the dynamics in plain FP32 geometry alone."""
    if precise:
        return float(K) * H * (n_sub * SUBSTEP + PER_DT_STEP + PER_DT_STEP_PRECISE)
    return float(K) * H * (n_sub * SUBSTEP_DYNAMICS + PER_DT_STEP)


def sample_bytes(K: int, D: int = 48) -> float:
    """K1: writes U[K][D] floats (reads D floats of mu); D = 48 knots, or 12 H
    direct targets."""
    return 4.0 * K * D + 4 * D


def update_bytes(K: int, D: int = 48) -> float:
    """K3/K4: reads L[K] and U[K][D]; writes the updated and the shifted mean
    and u0."""
    return 4.0 * K * (D + 1) + 4 * (D + D + 12)


def fp32_peak_tflops(sms: int = 152, mhz: float = 2070.0) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12
