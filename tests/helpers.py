"""Test helpers: map a workload onto the oracle's structures."""
import oracle as o

_BCS = {"periodic": o.BC_PERIODIC, "inlet": o.BC_INLET, "outlet": o.BC_OUTLET,
        "symmetry": o.BC_SYMMETRY, "noslip": o.BC_NOSLIP, "outlet_free": o.BC_OUTLET_FREE}
_KINDS = {"none": o.BODY_NONE, "disk": o.BODY_DISK, "naca": o.BODY_NACA}


def oracle_config(w):
    return o.make_config(w.nx, w.ny, bc=tuple(_BCS[b] for b in w.bc),
                         collision=o.BGK if w.collision == "bgk" else o.TRT,
                         forcing=o.FORCING_PAPER if w.forcing == "paper" else o.FORCING_SPLIT,
                         tau_plus=w.tau_plus, lambda_trt=w.lambda_trt, eta=w.eta, u_in=w.u_in,
                         body_force=w.body_force)


def oracle_body(w):
    b = w.body
    return o.make_body(_KINDS[b.kind], length=b.length, thickness=b.thickness, xg=b.x_c,
                       yg=b.y_c, theta=b.angle, pivot_frac=b.pivot_chord_frac,
                       moving=1 if b.moving else 0, density_ratio=b.density_ratio,
                       gravity=b.gravity, n_sim=b.n_sim_points)


def oracle_setup(w):
    """(cfg, body, chi, f0, sim points) of a workload in the oracle."""
    cfg, body = oracle_config(w), oracle_body(w)
    chi = o.raster(body, w.nx, w.ny)
    f = o.init(cfg, body, chi)
    pts = o.sim_points(body) if w.body.kind != "none" else None
    return cfg, body, chi, f, pts
