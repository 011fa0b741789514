"""Layout conversion between the element-major storage and the global subcell
grid (test infrastructure: oracle).

Storage (the library's layout): u[e][v][t], element e = ex + nx*(ey + ny*ez),
subcell t = ix + M*(iy + M*iz) (x fastest), v = 0..d+1 the conserved variable.
Global grid: U[v, gz, gy, gx] with g = e_axis*M + i_axis (x is the last axis).
"""
import numpy as np


def to_grid(u, dim, M, nel):
    """(E, nv, M^d) element-major array -> (nv, G_{d-1}, ..., G_0) global grid."""
    u = np.asarray(u)
    nv = u.shape[1]
    if dim == 2:
        nx, ny = nel[0], nel[1]
        x = u.reshape(ny, nx, nv, M, M)            # ey, ex, v, iy, ix
        x = x.transpose(2, 0, 3, 1, 4)             # v, ey, iy, ex, ix
        return np.ascontiguousarray(x.reshape(nv, ny * M, nx * M))
    nx, ny, nz = nel[0], nel[1], nel[2]
    x = u.reshape(nz, ny, nx, nv, M, M, M)         # ez, ey, ex, v, iz, iy, ix
    x = x.transpose(3, 0, 4, 1, 5, 2, 6)           # v, ez, iz, ey, iy, ex, ix
    return np.ascontiguousarray(x.reshape(nv, nz * M, ny * M, nx * M))


def to_elements(U, dim, M, nel):
    """Inverse of to_grid."""
    U = np.asarray(U)
    nv = U.shape[0]
    if dim == 2:
        nx, ny = nel[0], nel[1]
        x = U.reshape(nv, ny, M, nx, M).transpose(1, 3, 0, 2, 4)
        return np.ascontiguousarray(x.reshape(ny * nx, nv, M * M))
    nx, ny, nz = nel[0], nel[1], nel[2]
    x = U.reshape(nv, nz, M, ny, M, nx, M).transpose(1, 3, 5, 0, 2, 4, 6)
    return np.ascontiguousarray(x.reshape(nz * ny * nx, nv, M ** 3))


def sub_to_elements(S, dim, k, nel):
    """Per-sub-element scalar array (G_{d-1}/n, ..., G_0/n) with k = M/n sub-elements
    per axis and element -> (E, k^d) with the element's sub-elements x fastest."""
    S = np.asarray(S)
    if dim == 2:
        nx, ny = nel[0], nel[1]
        x = S.reshape(ny, k, nx, k).transpose(0, 2, 1, 3)
        return np.ascontiguousarray(x.reshape(ny * nx, k * k))
    nx, ny, nz = nel[0], nel[1], nel[2]
    x = S.reshape(nz, k, ny, k, nx, k).transpose(0, 2, 4, 1, 3, 5)
    return np.ascontiguousarray(x.reshape(nz * ny * nx, k ** 3))


def sub_from_elements(S, dim, k, nel):
    """Inverse of sub_to_elements."""
    S = np.asarray(S)
    if dim == 2:
        nx, ny = nel[0], nel[1]
        x = S.reshape(ny, nx, k, k).transpose(0, 2, 1, 3)
        return np.ascontiguousarray(x.reshape(ny * k, nx * k))
    nx, ny, nz = nel[0], nel[1], nel[2]
    x = S.reshape(nz, ny, nx, k, k, k).transpose(0, 3, 1, 4, 2, 5)
    return np.ascontiguousarray(x.reshape(nz * k, ny * k, nx * k))
