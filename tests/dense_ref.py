"""Brute-force dense solvers used only as test pins: the DG0 upwind SN and
collocation systems assembled as explicit matrices and solved directly."""
import numpy as np


def neighbours(nx, ny, ox, oy):
    """For each cell: the x-upwind and y-upwind cell index or -1 (inflow)."""
    sx = 1 if ox > 0 else -1
    sy = 1 if oy > 0 else -1
    ux = np.full(nx * ny, -1)
    uy = np.full(nx * ny, -1)
    for iy in range(ny):
        for ix in range(nx):
            c = iy * nx + ix
            jx, jy = ix - sx, iy - sy
            if 0 <= jx < nx:
                ux[c] = iy * nx + jx
            if 0 <= jy < ny:
                uy[c] = jy * nx + ix
    return ux, uy


def transport_block(nx, ny, hx, hy, ox, oy, sigma_t, psi_edge):
    """Matrix T and inflow vector g with T psi = src + g for one direction."""
    N = nx * ny
    ax, ay = abs(ox) / hx, abs(oy) / hy
    ux, uy = neighbours(nx, ny, ox, oy)
    T = np.diag(sigma_t + ax + ay)
    g = np.zeros(N)
    pin_x = psi_edge[0] if ox > 0 else psi_edge[1]
    pin_y = psi_edge[2] if oy > 0 else psi_edge[3]
    for c in range(N):
        if ux[c] >= 0:
            T[c, ux[c]] -= ax
        else:
            g[c] += ax * pin_x
        if uy[c] >= 0:
            T[c, uy[c]] -= ay
        else:
            g[c] += ay * pin_y
    return T, g


def sn_dense(p, coef, psi0, ox, oy, w):
    """Solve the full discrete SN system (all angles coupled through phi)."""
    nx, ny = p.nx, p.ny
    N, K = nx * ny, len(w)
    hx, hy = p.lx / nx, p.ly / ny
    A = np.zeros((N * K, N * K))
    b = np.zeros(N * K)
    inv_cdt = 1.0 / (p.c * p.dt)
    for k in range(K):
        T, g = transport_block(nx, ny, hx, hy, ox[k], oy[k], coef["sigma_t"], p.psi_edge)
        A[k * N:(k + 1) * N, k * N:(k + 1) * N] += T
        for kp in range(K):
            A[k * N:(k + 1) * N, kp * N:(kp + 1) * N] -= np.diag(coef["sigma_s"] / (4 * np.pi) * w[kp])
        b[k * N:(k + 1) * N] = coef["q"] + inv_cdt * psi0[:, k] + g
    return np.linalg.solve(A, b).reshape(K, N).T


def sn_dense_reflect(p, coef, psi0, ox, oy, w, reflect, mirror_x, mirror_y):
    """The full SN system with reflective edges coupled implicitly: a
    direction entering through a reflective edge takes, in the same cell, the
    value of its mirror direction (mirror_x[k], mirror_y[k])."""
    nx, ny = p.nx, p.ny
    N, K = nx * ny, len(w)
    hx, hy = p.lx / nx, p.ly / ny
    A = np.zeros((N * K, N * K))
    b = np.zeros(N * K)
    inv_cdt = 1.0 / (p.c * p.dt)
    for k in range(K):
        edge = list(p.psi_edge)
        ex, ey = (0 if ox[k] > 0 else 1), (2 if oy[k] > 0 else 3)
        if reflect[ex]:
            edge[ex] = 0.0
        if reflect[ey]:
            edge[ey] = 0.0
        T, g = transport_block(nx, ny, hx, hy, ox[k], oy[k], coef["sigma_t"], edge)
        A[k * N:(k + 1) * N, k * N:(k + 1) * N] += T
        ax, ay = abs(ox[k]) / hx, abs(oy[k]) / hy
        for iy in range(ny):
            if reflect[ex]:
                c = iy * nx + (0 if ex == 0 else nx - 1)
                A[k * N + c, mirror_x[k] * N + c] -= ax
        for ix in range(nx):
            if reflect[ey]:
                c = (0 if ey == 2 else ny - 1) * nx + ix
                A[k * N + c, mirror_y[k] * N + c] -= ay
        for kp in range(K):
            A[k * N:(k + 1) * N, kp * N:(kp + 1) * N] -= np.diag(coef["sigma_s"] / (4 * np.pi) * w[kp])
        b[k * N:(k + 1) * N] = coef["q"] + inv_cdt * psi0[:, k] + g
    return np.linalg.solve(A, b).reshape(K, N).T
