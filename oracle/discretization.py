"""Oracle discretization: voxelised cubic meta-atoms with rooftop currents.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper expands J in loop/star functions on a finite-element mesh (Sec. 3,
eq. eqn04).  The workloads here are cubes split into n_v^3 voxels with one
div-conforming rooftop per voxel face, boundary faces included, so an atom
carries 3 (n_v+1) n_v^2 unknowns.  Unknowns are ordered atom by atom
(Sec. 4, eq. bp); inside an atom: x-faces, then y-faces, then z-faces, each in
lexicographic (i, j, k) order where the normal index runs over 0..n_v.

Rooftop on a face with normal e_d at coordinate f_d (voxel size h):
    w = h^-2 (1 - |r_d - f_d| / h) e_d      on the (one or two) voxels beside it.
On the voxel below the face (r_d < f_d) the profile is xi_d (local coordinate
0..1 from the voxel's low side); on the voxel above it is 1 - xi_d.
Its distributional divergence (the charge density times -j omega) is
+h^-3 on the voxel below, -h^-3 on the voxel above, and for a face on the
cube boundary a sheet of -h^-2 (upper boundary) or +h^-2 (lower boundary) on
the face itself, so that it integrates to zero.
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass
class AtomMesh:
    """Local (corner-at-origin) mesh of one atom type."""
    side: float
    nv: int
    h: float = field(init=False)
    vox_idx: np.ndarray = field(init=False)      # (nvox, 3) integer voxel indices
    face_dir: np.ndarray = field(init=False)     # (nf,)
    face_idx: np.ndarray = field(init=False)     # (nf, 3) integer indices
    face_lo_vox: np.ndarray = field(init=False)  # voxel below the face or -1
    face_hi_vox: np.ndarray = field(init=False)  # voxel above the face or -1
    face_sheet: np.ndarray = field(init=False)   # surface element index or -1
    face_sheet_sign: np.ndarray = field(init=False)  # +1 lower boundary, -1 upper, 0 interior
    surf_face: np.ndarray = field(init=False)    # face index of each surface element

    def __post_init__(self):
        n = self.nv
        self.h = self.side / n
        self.vox_idx = np.array([(i, j, k) for i in range(n) for j in range(n) for k in range(n)])
        dirs, idxs, lo, hi, sheet, ssign, surf = [], [], [], [], [], [], []
        for d in range(3):
            ranges = [range(n), range(n), range(n)]
            ranges[d] = range(n + 1)
            for i in ranges[0]:
                for j in ranges[1]:
                    for k in ranges[2]:
                        ijk = [i, j, k]
                        f = len(dirs)
                        dirs.append(d)
                        idxs.append(ijk)
                        m = ijk[d]
                        below = list(ijk); below[d] = m - 1
                        lo.append(self.voxel_number(below) if m >= 1 else -1)
                        hi.append(self.voxel_number(ijk) if m <= n - 1 else -1)
                        if m == 0 or m == n:
                            sheet.append(len(surf)); surf.append(f)
                            ssign.append(+1 if m == 0 else -1)
                        else:
                            sheet.append(-1); ssign.append(0)
        self.face_dir = np.array(dirs)
        self.face_idx = np.array(idxs)
        self.face_lo_vox = np.array(lo)
        self.face_hi_vox = np.array(hi)
        self.face_sheet = np.array(sheet)
        self.face_sheet_sign = np.array(ssign)
        self.surf_face = np.array(surf, dtype=int)

    def voxel_number(self, ijk):
        n = self.nv
        return (ijk[0] * n + ijk[1]) * n + ijk[2]

    @property
    def n_faces(self):
        return len(self.face_dir)

    @property
    def n_vox(self):
        return len(self.vox_idx)

    def voxel_box(self, v, origin):
        lo = origin + self.h * self.vox_idx[v]
        return lo, lo + self.h

    def surf_rect(self, s, origin):
        """(axis, coord, lo, hi) of surface element s."""
        f = self.surf_face[s]
        d = self.face_dir[f]
        ijk = self.face_idx[f]
        lo = origin + self.h * ijk.astype(float)
        hi = lo + self.h
        hi[d] = lo[d]
        return d, lo[d], lo, hi

    def face_voxels(self, f):
        """[(voxel, profile)] with profile +1 = xi_d (voxel below), -1 = 1 - xi_d (above)."""
        out = []
        if self.face_lo_vox[f] >= 0:
            out.append((self.face_lo_vox[f], +1))
        if self.face_hi_vox[f] >= 0:
            out.append((self.face_hi_vox[f], -1))
        return out

    def face_charges(self, f):
        """Volume pieces [(voxel, density)] and sheet pieces [(surf, density)] of div w_f."""
        h = self.h
        vol = []
        if self.face_lo_vox[f] >= 0:
            vol.append((self.face_lo_vox[f], +h ** -3))
        if self.face_hi_vox[f] >= 0:
            vol.append((self.face_hi_vox[f], -h ** -3))
        sur = []
        if self.face_sheet[f] >= 0:
            sur.append((self.face_sheet[f], self.face_sheet_sign[f] * h ** -2))
        return vol, sur


@dataclass
class Problem:
    """Array of cubic meta-atoms (units: lengths in the same unit as the wavelength).

    centres: (N, 3) atom centres; types: (N,) type index; sides, nvs, eps: per type.
    """
    centres: np.ndarray
    types: np.ndarray
    sides: np.ndarray
    nvs: np.ndarray
    eps: np.ndarray
    wavelength: float

    def __post_init__(self):
        self.centres = np.asarray(self.centres, dtype=np.float64)
        self.types = np.asarray(self.types, dtype=int)
        self.meshes = [AtomMesh(float(s), int(n)) for s, n in zip(self.sides, self.nvs)]
        self.k = 2.0 * np.pi / self.wavelength
        sizes = np.array([self.meshes[t].n_faces for t in self.types])
        self.offsets = np.concatenate([[0], np.cumsum(sizes)])

    @property
    def n_atoms(self):
        return len(self.types)

    @property
    def n(self):
        return int(self.offsets[-1])

    def origin(self, i):
        return self.centres[i] - 0.5 * self.sides[self.types[i]]

    def mesh(self, i):
        return self.meshes[self.types[i]]
