"""Diagnostics log of a run: the 16 FP64 diagnostics of ``vefd_diagnostics``
every ``every`` steps, written as CSV rows (host-side bookkeeping; every step
and every reduction runs in the library's kernels).

Columns: step, mass_A, mass_B, px, py, pz, sigma_xy, N1, max_trC_over_L2,
max_u, area_mid_plane, D, theta, centroid_x, centroid_y, volume, trace_sigma_m3,
mass_drift (the largest relative change of a component mass since the start).
"""
import csv

COLUMNS = ["step", "mass_A", "mass_B", "px", "py", "pz", "sigma_xy", "N1", "max_trC_over_L2", "max_u",
           "area_mid_plane", "D", "theta", "centroid_x", "centroid_y", "volume", "trace_sigma_m3", "mass_drift"]


def run_logged(lat, nsteps, every, path=None, status_check=True):
    """Steps `lat` (a vefd.Lattice) nsteps times, taking the diagnostics before
    the first step and after every `every` steps (and after the last); returns
    the rows, and writes them to `path` as CSV when given.  With status_check
    the guard word is read at every row and a set bit stops the run with
    vefd.VefdError (status ERR_UNSTABLE or ERR_TIMEOUT)."""
    from . import vefd
    if every < 1 or nsteps < 0:
        raise ValueError("every must be >= 1 and nsteps >= 0")
    rows = []
    d0 = lat.diagnostics()
    m0 = [d0[0], d0[1]]

    def row(step, d):
        drift = max(abs(d[k] / m0[k] - 1.0) if m0[k] else 0.0 for k in (0, 1))
        rows.append([int(step)] + [float(v) for v in d] + [drift])

    row(lat.steps_done, d0)
    done = 0
    while done < nsteps:
        n = min(every, nsteps - done)
        lat.step(n)
        done += n
        row(lat.steps_done, lat.diagnostics())
        if status_check:
            bits = lat.status()
            if bits:
                if path:
                    _write(path, rows)
                raise vefd.VefdError(vefd.ERR_TIMEOUT if bits & vefd.ST_TIMEOUT else vefd.ERR_UNSTABLE,
                                     "guard bits %#x at step %d" % (bits, lat.steps_done))
    if path:
        _write(path, rows)
    return rows


def _write(path, rows):
    with open(path, "w", newline="") as fh:
        w = csv.writer(fh)
        w.writerow(COLUMNS)
        w.writerows(rows)
