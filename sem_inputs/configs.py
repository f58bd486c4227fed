"""Named mesh descriptors for the workloads.

The paper's pipe meshes (Sec. 4.2: 237,120 and 853,632 elements) are not
available; synthetic O-grid pipes of matching regime stand in for them
(E = 4096 sits in the 2000-5000 elements-per-GPU strong-scaling limit of
Sec. 7; E = 262,144 and 1,048,576 are whole-GPU loads).  For the pipe, the
cross-section holds nc (nc + 4 nr) elements, so the counts are powers of two.
"""

MESHES = {
    # 3D Poisson on the unit cube, 4x4x4 affine elements, N = 7.
    "box4_n7": dict(kind="box", nx=4, ny=4, nz=4, N=7, lx=1.0, ly=1.0, lz=1.0),
    # Straight pipe R = 1, L = 8, O-grid, wall clustering beta = 2, periodic in z.
    "pipe4096_n7": dict(kind="pipe", nc=8, nr=2, nzp=32, N=7, R=1.0, L=8.0, a=0.5, beta=2.0, periodic=True),
    "pipe262144_n7": dict(kind="pipe", nc=16, nr=4, nzp=512, N=7, R=1.0, L=8.0, a=0.5, beta=2.0, periodic=True),
    # same cross-section and element shape as pipe262144_n7, 1/8 of the length (profiling size, > L2)
    "pipe32768_n7": dict(kind="pipe", nc=16, nr=4, nzp=64, N=7, R=1.0, L=1.0, a=0.5, beta=2.0, periodic=True),
    "pipe1048576_n7": dict(kind="pipe", nc=32, nr=8, nzp=512, N=7, R=1.0, L=8.0, a=0.5, beta=2.0, periodic=True),
    "pipe131072_n11": dict(kind="pipe", nc=16, nr=4, nzp=256, N=11, R=1.0, L=8.0, a=0.5, beta=2.0, periodic=True),
}


def mesh_desc(name, **override):
    d = dict(MESHES[name])
    d.update(override)
    return d


def elements_of(desc):
    if desc["kind"] == "box":
        return desc["nx"] * desc["ny"] * desc["nz"]
    if desc["kind"] == "pipe":
        return desc["nc"] * (desc["nc"] + 4 * desc["nr"]) * desc["nzp"]
    raise ValueError(desc["kind"])
