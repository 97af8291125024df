"""Plain definitions used by the oracle pins: raw and central moments of a
population vector (Eq. 19 / Eq. 21 / Eq. 37 / Eq. 38 and their 3D analogues),
the orthogonal bases of Eq. 17 and Eq. 35, and Maxwellian central-moment
values.  Written independently of the oracle, from the definitions alone."""
import numpy as np

D2Q9_E = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0],
                   [1, 1, 0], [-1, 1, 0], [-1, -1, 0], [1, -1, 0]], dtype=float)
D2Q5_E = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]], dtype=float)
D3Q27_E = np.array([[a % 3 - 1, (a // 3) % 3 - 1, a // 9 - 1] for a in range(27)], dtype=float)

# Appendix A, Eq. a1
D3Q15_E = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                    [1, 1, 1], [-1, 1, 1], [1, -1, 1], [-1, -1, 1], [1, 1, -1], [-1, 1, -1], [1, -1, -1],
                    [-1, -1, -1]], dtype=float)

W_D2Q9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W_D2Q5 = np.array([1 / 3] + [1 / 6] * 4)
W_D3Q27 = np.array([np.prod([2 / 3 if c == 0 else 1 / 6 for c in e]) for e in D3Q27_E])
# textbook D3Q15 weights (rest 2/9, axes 1/9, corners 1/72)
W_D3Q15 = np.array([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)


def central(f, E, u, a, b, c=0):
    """sum_alpha f_alpha (e_x - u_x)^a (e_y - u_y)^b (e_z - u_z)^c."""
    return float(np.sum(f * (E[:, 0] - u[0]) ** a * (E[:, 1] - u[1]) ** b * (E[:, 2] - u[2]) ** c))


def raw(f, E, a, b, c=0):
    return float(np.sum(f * E[:, 0] ** a * E[:, 1] ** b * E[:, 2] ** c))


def maxwell_central(rho, a, b, c=0):
    """Central moments of a Maxwellian with c_s^2 = 1/3 (Eq. 20, Eq. 39)."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    v = rho
    for n in (a, b, c):
        if n == 2:
            v /= 3.0
    return v


def K_d2q9():
    """Columns |K_0>..|K_8> of Eq. 17."""
    ex, ey = D2Q9_E[:, 0], D2Q9_E[:, 1]
    one = np.ones(9)
    return np.stack([one, ex, ey, 3 * (ex ** 2 + ey ** 2) - 4 * one, ex ** 2 - ey ** 2, ex * ey,
                     -3 * ex ** 2 * ey + 2 * ey, -3 * ex * ey ** 2 + 2 * ex,
                     9 * ex ** 2 * ey ** 2 - 6 * (ex ** 2 + ey ** 2) + 4 * one], axis=1)


def L_d2q5():
    """Columns |L_0>..|L_4> of Eq. 35."""
    ex, ey = D2Q5_E[:, 0], D2Q5_E[:, 1]
    one = np.ones(5)
    return np.stack([one, ex, ey, 5 * (ex ** 2 + ey ** 2) - 4 * one, ex ** 2 - ey ** 2], axis=1)


def K_d3q15():
    """Columns |K_0>..|K_14> of Eq. 2A."""
    ex, ey, ez = D3Q15_E[:, 0], D3Q15_E[:, 1], D3Q15_E[:, 2]
    one = np.ones(15)
    e2 = ex ** 2 + ey ** 2 + ez ** 2
    return np.stack([one, ex, ey, ez, ex * ey, ex * ez, ey * ez, ex ** 2 - ey ** 2, e2 - 3 * ez ** 2,
                     e2 - 2 * one, 5 * ex * e2 - 13 * ex, 5 * ey * e2 - 13 * ey, 5 * ez * e2 - 13 * ez,
                     ex * ey * ez,
                     30 * (ex ** 2 * ey ** 2 + ex ** 2 * ez ** 2 + ey ** 2 * ez ** 2) - 40 * e2 + 32 * one], axis=1)
