"""Uniform finite-volume grid and metric for the oracle (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper meshes a 2D-axisymmetric slice with an unstructured mesh (Sec. 3.1.1);
here the domain is a uniform grid, either axisymmetric r-z (axis 0 = r, axis 1 =
z, one cell in the third direction, everything per radian) or 3D Cartesian.

Arrays use shape (n0, n1, n2) (index 0 fastest in the flattened, Fortran-order
vector).  A face array for direction a has n_a + 1 entries along a.

Boundary kinds per side (Table tableboundary):
  AXIS   symmetry axis r = 0 (zero face area)
  WALL   outerWall: no slip, zero gradient of T and omega, Neumann pressure
  OPEN   natural-convection inlet / outlet: inletOutlet T, omega, u; p_rgh = p_ext
  FORCED forced-convection inlet: fixed u, T, omega; Neumann pressure
"""
import numpy as np

AXIS, WALL, OPEN, FORCED = 0, 1, 2, 3


class Grid:
    def __init__(self, cfg):
        self.axisym = cfg["geom"] == 0
        n = list(cfg["n"])
        if self.axisym:
            n[2] = 1
        self.n = tuple(int(v) for v in n)
        self.act = [0, 1] if self.axisym else [0, 1, 2]
        self.h = [cfg["L"][a] / self.n[a] if a in self.act else 1.0 for a in range(3)]
        self.hmin = min(self.h[a] for a in self.act)
        self.s = 1 if self.axisym else 2          # streamwise (gravity / inflow) axis
        inlet = FORCED if cfg["bc_mode"] == 1 else OPEN
        if self.axisym:
            self.bc = [[AXIS, WALL], [inlet, OPEN], [WALL, WALL]]
        else:
            self.bc = [[WALL, WALL], [WALL, WALL], [inlet, OPEN]]
        # cell-centre and face coordinates along each axis
        self.xc = [(np.arange(self.n[a]) + 0.5) * self.h[a] for a in range(3)]
        self.xf = [np.arange(self.n[a] + 1) * self.h[a] for a in range(3)]
        self.V = self._cell_volume()
        self.A = [self._face_area(a) if a in self.act else None for a in range(3)]

    # -- broadcasting helpers ------------------------------------------------
    @staticmethod
    def along(v, a):
        """The 1D array v as a (3D) array varying along axis a only, for broadcasting."""
        shape = [1, 1, 1]
        shape[a] = v.shape[0]
        return v.reshape(shape)

    def _cell_volume(self):
        h = self.h
        if self.axisym:
            r = self.along(self.xc[0], 0)
            return np.broadcast_to(r * h[0] * h[1], self.n).copy()
        return np.full(self.n, h[0] * h[1] * h[2])

    def _face_area(self, a):
        h = self.h
        shape = list(self.n)
        shape[a] += 1
        if self.axisym:
            if a == 0:
                r = self.along(self.xf[0], 0)          # face radius i*dr
                return np.broadcast_to(r * h[1], shape).copy()
            r = self.along(self.xc[0], 0)              # z-face: centre radius
            return np.broadcast_to(r * h[0], shape).copy()
        return np.full(shape, h[0] * h[1] * h[2] / h[a])

    def area_normal(self, a, rloc):
        """Area of a face normal to axis a located at radial coordinate rloc
        (axisymmetric; per radian) or the Cartesian face area."""
        h = self.h
        if self.axisym:
            return rloc * (h[1] if a == 0 else h[0])
        return h[0] * h[1] * h[2] / h[a]

    def ncell(self):
        """Number of cells."""
        return self.n[0] * self.n[1] * self.n[2]

    def lin(self, i, j, k):
        """Linear cell index, i fastest."""
        return i + self.n[0] * (j + self.n[1] * k)
