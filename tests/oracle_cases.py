"""Oracle-side construction of the workloads of paper_2004_05197_gb300.workloads."""
from oracle.assembly import Space
from oracle.geometry import AnnulusQuarter, BsplineThetaCoef, ConstCoef, CubeSinePerturbed, IdentityMap, SinCosCoef
from oracle.surrogate import Surrogate


def oracle_space(w):
    geo = {"annulus": AnnulusQuarter(), "cube": CubeSinePerturbed(0.1),
           "identity": IdentityMap(w["dim"])}[w["map"]]
    if w["coef"] == "const":
        coef = ConstCoef(1.0)
    elif w["coef"] == "sincos":
        coef = SinCosCoef(0.5)
    else:
        from paper_2004_05197_gb300.workloads import theta_for
        coef = BsplineThetaCoef(theta_for(w), 3)
    return Space(w["dim"], w["p"], w["n_el"], geo, coef)


def oracle_surrogate(w, M=None):
    sp = oracle_space(w)
    return sp, Surrogate(sp, w["q"], w["M"] if M is None else M)
