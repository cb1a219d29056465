"""Recycling-strategy acronyms of Table 1: VecType-Size(Side)[-NSC].

VecType: Ritz (Ritz vectors), HRitz (harmonic Ritz vectors), RGen (Ritz generalized
singular vectors); Size: S (smallest), L (largest), M (half of each); Side (RGen only):
R (right, W X), L (left, W V_H), M (their average).  A trailing "-NSC" selects the
hypergradient-error stopping rule of Section 4.  "none" means plain CG.  The
full-space variants Eig-S and GSVD-L(R) need the dense Hessian and are not offered.
"""
from __future__ import annotations

import re
from dataclasses import dataclass

_RE = re.compile(r"^(Ritz|HRitz|RGen)-([SLM])(?:\(([RLM])\))?(-NSC)?$")


@dataclass(frozen=True)
class Strategy:
    kind: str = "none"       # "none" | "ritz" | "hritz" | "rgsv"
    size: str = "S"
    side: str = "R"
    nsc: bool = False

    @property
    def recycles(self) -> bool:
        return self.kind != "none"

    def acronym(self) -> str:
        if self.kind == "none":
            return "none"
        name = {"ritz": "Ritz", "hritz": "HRitz", "rgsv": "RGen"}[self.kind]
        s = f"{name}-{self.size}"
        if self.kind == "rgsv":
            s += f"({self.side})"
        return s + ("-NSC" if self.nsc else "")


def parse(acronym: str) -> Strategy:
    if acronym.strip().lower() in ("none", "cg", ""):
        return Strategy()
    m = _RE.match(acronym.strip())
    if not m:
        raise ValueError(f"not a recycling strategy acronym: {acronym!r}")
    vec, size, side, nsc = m.groups()
    kind = {"Ritz": "ritz", "HRitz": "hritz", "RGen": "rgsv"}[vec]
    if kind != "rgsv" and side is not None:
        raise ValueError(f"{vec} takes no side: {acronym!r}")
    if kind == "rgsv" and side is None:
        raise ValueError(f"RGen needs a side, e.g. RGen-L(R): {acronym!r}")
    if nsc and kind != "rgsv":
        raise ValueError(f"the NSC stopping rule needs Ritz generalized singular vectors: {acronym!r}")
    return Strategy(kind, size, side or "R", bool(nsc))
