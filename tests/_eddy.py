"""The 2D eddy-current example of Sec. 4.2 (unit square, kappa = mu = 1,
Neumann boundary): the exact solution E (zero on Omega_2 = {x1 <= x2}), its
curl, and the right-hand side F = curlv curl E + E, written out by the chain
rule. With a = x1 - x2, b = x1 - 1 and phi = x2 a^2 b^2 on Omega_1:
  E = (sin(2 pi x1) + 2 pi cos(2 pi x1) a, sin(phi) - sin(2 pi x1)),
  curl E = dE2/dx1 - dE1/dx2 = g cos(phi), g = d phi / dx1 = 2 x2 a b (a + b),
  curlv s = (ds/dx2, -ds/dx1).
Evaluated elementwise: the mesh's "/" diagonals follow x1 = x2, so an element
lies in one part; `inside` says which (from its centroid)."""
import numpy as np


def exact(x1, x2, inside):
    """E, curl E at points (arrays), zero where inside is False."""
    tp = 2.0 * np.pi
    a, b = x1 - x2, x1 - 1.0
    phi = x2 * a * a * b * b
    g = 2.0 * x2 * a * b * (a + b)
    E1 = np.sin(tp * x1) + tp * np.cos(tp * x1) * a
    E2 = np.sin(phi) - np.sin(tp * x1)
    curl = g * np.cos(phi)
    return np.where(inside, E1, 0.0), np.where(inside, E2, 0.0), np.where(inside, curl, 0.0)


def rhs(x1, x2, inside):
    """F = curlv curl E + E (kappa = mu = 1)."""
    a, b = x1 - x2, x1 - 1.0
    phi = x2 * a * a * b * b
    g = 2.0 * x2 * a * b * (a + b)
    dphi2 = a * b * b * (a - 2.0 * x2)
    dg1 = 2.0 * x2 * (a * a + 4.0 * a * b + b * b)
    dg2 = 2.0 * a * b * (a + b) - 2.0 * x2 * b * (2.0 * a + b)
    dc1 = dg1 * np.cos(phi) - g * g * np.sin(phi)
    dc2 = dg2 * np.cos(phi) - g * np.sin(phi) * dphi2
    E1, E2, _ = exact(x1, x2, inside)
    return np.where(inside, dc2 + E1, 0.0), np.where(inside, -dc1 + E2, 0.0)
