"""A sequence of trial potentials fitted to the same data (Section 4): the
models of all trial potentials advanced together in one batch, and their
final chi^2 and merit F compared (the mass-model selection of that
section)."""
from . import m2m as B


def potential_scan(problems, nsteps, precision="fp32c", device="cuda:0", targets=None, tune_steps=0):
    """Fit every problem (one per trial potential, the same observables) to
    the same data for nsteps M2M steps in one batch.

    targets: the observed values Y (with the error model of the inputs);
    None observes the target galaxy of problems[0] with the library.
    Returns (records, best): the last record of every model (step, chi2,
    chi2_raw, S, sum_w, F, max_abs_dt) and the index of the lowest chi2."""
    if targets is None:
        targets = B.observe_targets(problems[0], precision, device)
    models = [P.with_targets(targets) for P in problems]
    bt = B.m2m_batch_init(precision, models, device)
    try:
        if tune_steps:
            bt.m2m_batch_autotune(tune_steps)
        bt.m2m_batch_step(nsteps)
        records = bt.m2m_batch_get_records()
    finally:
        bt.m2m_batch_free()
    best = min(range(len(records)), key=lambda m: records[m]["chi2"])
    return records, best
