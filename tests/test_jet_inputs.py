"""The planar jet's inputs (workloads.jet_2d) against the geometry the
paper states (Section "Two Dimensional Jet Buckling"): the container is the
circle of radius 0.4 at (0.5, 0.5) below the ceiling y = 0.8, every row of
v faces over the opening carries exactly the inflow flux D U, the u faces
carry no inflow, and the source region is the opening."""
import numpy as np

from paper_1010_2832_gb300 import workloads as W


def test_jet_geometry_and_inflow():
    n = 150
    wl = W.jet_2d(n)
    h = wl.h
    J = W.JET2D
    X = W.lattice_points(wl.n, h, wl.origin)
    r = np.hypot(X[0] - 0.5, X[1] - 0.5)
    fluid = wl.phi_solid > 0
    assert np.all(r[fluid] < 0.4) and np.all(X[1][fluid] < 0.8)
    assert np.all(fluid[(r < 0.39) & (X[1] < 0.79)])
    P = W.sample_points("v", wl.n, h, wl.origin)
    above = P[1][:, 0] >= 0.8 - h / 4
    flux = wl.u_bc[1].sum(axis=1) * h
    assert np.allclose(flux[above], J["width"] * J["U"], rtol=1e-12)
    assert np.all(flux[~above] == 0) and np.all(wl.u_bc[0] == 0)
    src = W.jet_2d_source(n)
    inside = (np.abs(X[0] - 0.5) < 0.03 - 1e-9) & (X[1] > 0.8 + 1e-9)
    outside = (np.abs(X[0] - 0.5) > 0.03 + 1e-9) | (X[1] < 0.8 - 1e-9)
    assert np.all(src[inside] < 0) and np.all(src[outside] > 0)
    stub = wl.phi_liquid < 0
    assert np.all(stub[inside]) and stub.sum() > inside.sum()
