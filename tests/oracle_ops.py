"""Flat-vector adapters around the FP64 oracle, in the C ABI's vector layouts."""
import numpy as np

import oracle as O


def nodes_split(geo, v):
    out, off = [], 0
    for W in geo.wfs:
        k = (W["N"] + 1) ** 2
        out.append(np.asarray(v[off:off + k], float).reshape(W["N"] + 1, W["N"] + 1))
        off += k
    return out


def n_nodes(geo):
    return sum((W["N"] + 1) ** 2 for W in geo.wfs)


def project(geo, phi_flat):
    phis = geo.split(phi_flat)
    return np.concatenate([O.project(geo, g, phis).ravel() for g in range(len(geo.wfs))])


def project_adj(geo, v):
    out = [np.zeros((L["n"], L["n"])) for L in geo.layers]
    for g, vg in enumerate(nodes_split(geo, v)):
        for l, y in enumerate(O.project_adj(geo, g, vg)):
            out[l] += y
    return geo.join(out)


def slopes(geo, v):
    return np.concatenate([O.sh_slopes(geo, g, vg) for g, vg in enumerate(nodes_split(geo, v))])


def slopes_adj(geo, s):
    return np.concatenate([O.sh_slopes_adj(geo, g, s[W["soff"]:W["soff"] + W["ns"]]).ravel()
                           for g, W in enumerate(geo.wfs)])


def noise_weight(geo, s):
    return np.concatenate([O.noise_weight(geo, g, s[W["soff"]:W["soff"] + W["ns"]])
                           for g, W in enumerate(geo.wfs)])


def dwt(geo, phi_flat):
    return O.W_fwd(geo, geo.split(phi_flat))


def idwt(geo, c):
    return geo.join(O.W_inv(geo, c))


def forward(geo, phi_flat):
    return O.forward_model(geo, geo.split(phi_flat))


def forward_adj(geo, s):
    return geo.join(O.forward_model_adj(geo, s))
