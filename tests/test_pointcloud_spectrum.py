"""The point-cloud configuration's operator is spectrally unstable (a CPU
reproduction of the finding the stepping reports rest on).

Section 5 ties stable time stepping to the eigenvalues of L_X lying in the
left half-plane, and Section 7 smooths the normals of scanned point clouds
before it builds operators on them.  The 2M-node point-cloud configuration
keeps raw 20-nearest-neighbour PCA normals and a Gaussian tangent jitter of
0.25 h.  On a 2,000-node version (n = 31, IMQ, kappa_T = 1e12, the oracle's
eps search) the dense spectrum of the oracle's L_X reaches further into
the right half-plane (max Re ~ +5.8e5) than into the left (min Re ~ -2.6e5),
while the same surface sampled without jitter and with analytic normals has
a positive part some 600 times smaller (max Re ~ +960 against min Re
~ -1600; the conical points of r = 1 + 0.1 sin 3theta cos 4phi at the poles
leave it a little) -- enough to make Gray-Scott stepping blow up at 2M nodes
as well -- and the smooth unit sphere (Fibonacci nodes, exact normals) has
its spectrum in the closed left half-plane (max Re at rounding level, the
constant mode), which is why it is the stable stand-in of the 2M-node
Gray-Scott run.  The implicit Gray-Scott system (I - dt delta L) of the
point cloud is therefore not the stable one BiCGSTAB is meant for."""
import numpy as np

from oracle import operator as oop
from oracle import weights as ow
from paper_1404_0812_gb300 import workloads as W


def _spectrum(ns):
    op = oop.build_operator(ns.X, ns.normals, 31, ow.IMQ, kappa_T=1e12)
    return np.linalg.eigvals(oop.dense(op, ns.N))


def test_pointcloud_spectrum_right_half_plane():
    N = 2000
    cloud = W.bumpy_sphere(N, jitter=0.25, seed=4, normals="pca")
    smooth = W.bumpy_sphere(N, jitter=0.0, seed=4, normals="analytic")
    lc, ls = _spectrum(cloud), _spectrum(smooth)
    scale_c, scale_s = np.abs(lc.real).max(), np.abs(ls.real).max()
    print(f"point cloud: max Re {lc.real.max():.4g}, min Re {lc.real.min():.4g}; "
          f"analytic: max Re {ls.real.max():.4g}, min Re {ls.real.min():.4g}")
    # the point cloud: the right half-plane part is as large as the left one
    assert lc.real.max() > 0.5 * abs(lc.real.min())
    # the smooth surface: mostly in the left half-plane, its positive part
    # two orders of magnitude below the point cloud's
    assert ls.real.max() < abs(ls.real.min())
    assert lc.real.max() > 100 * max(ls.real.max(), 1.0)
    assert scale_c > scale_s
    sphere = _spectrum(W.fibonacci_sphere(N))
    print(f"unit sphere: max Re {sphere.real.max():.4g}, min Re {sphere.real.min():.4g}")
    assert sphere.real.max() < 1e-8 * abs(sphere.real.min())
