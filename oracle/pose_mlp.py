"""Oracle of the paper's pose parameterisation (Section 3, Pose Refinement, Eq. 3, and the
optimiser of Implementation Details): plain numpy in FP64, for tests only.

    P_i^s = phi(P_i^0 + MLP(P_i^0)) + [0 | delta_i]

P^0 is the flattened initial 3x4 pose [R | t] (world -> camera, row-major, 12 values).  The
MLP has six linear layers of hidden width 128 (12 -> 128 -> 128 -> 128 -> 128 -> 128 -> 12),
ReLU after the first five and a skip connection after the third (the first layer's output
added to the third's).  phi is Gram-Schmidt on the 6D representation of Zhou et al. (the first
two columns of the 3x3 block); the translation passes through and delta_i is added.  The MLP
is shared by the views of one scene; delta is per view.

The parameterisation acts on the scene at unit scale (the paper's inputs are 3D foundation
model outputs, which are normalised): with s the RMS distance of the P^0 camera centres from
their centroid, the MLP sees P^0 with its translation divided by s, and its translation output
and delta are multiplied by s.  P_i^s = [phi(R' ) | t_i^0 + s (y_t + delta_i)].

Gradients come from the objective's left-perturbation gradient G_i = (g_v, g_w) of each pose
(translation first), turned into Euclidean derivatives of the pose entries, then back through
phi and the MLP.  AdamW (decoupled weight decay) with the learning-rate schedule of the paper:
a linear warm-up to lr_max over the first steps, then cosine decay to 0 at the last step.

Parameter layout (one flat float vector per scene): W1 (128x12, row-major [out][in]), b1 (128),
W2..W5 (128x128), b2..b5 (128), W6 (12x128), b6 (12): 69260 values.

This module is test infrastructure: only tests, the package's smoke check and the benchmark's
CPU baseline may import it."""
import numpy as np

HID = 128
DIMS = [(HID, 12), (HID, HID), (HID, HID), (HID, HID), (HID, HID), (12, HID)]
N_PARAMS = sum(o * i + o for o, i in DIMS)  # 69260


def unpack(theta):
    """Views (W, b) per layer into the flat parameter vector."""
    theta = np.asarray(theta)
    out, k = [], 0
    for o, i in DIMS:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def mlp_forward(theta, x):
    """x: (n, 12) -> y (n, 12) and the cache for the backward pass (pre-activations z_l and
    layer inputs a_{l-1})."""
    L = unpack(theta)
    a = [np.asarray(x, dtype=np.float64)]
    z = []
    h = a[0]
    h1 = None
    for l, (W, b) in enumerate(L):
        zl = h @ W.T + b
        z.append(zl)
        if l == 5:
            return zl, (a, z)
        h = np.maximum(zl, 0.0)
        if l == 0:
            h1 = h
        if l == 2:
            h = h + h1  # skip connection after the third layer
        a.append(h)


def mlp_backward(theta, cache, dy):
    """dL/dy (n, 12) -> dL/dtheta (flat) and dL/dx."""
    L = unpack(theta)
    a, z = cache
    grads = [None] * 6
    d = np.asarray(dy, dtype=np.float64)  # dL/dz_6
    dskip = None
    for l in range(5, -1, -1):
        W, _ = L[l]
        grads[l] = (d.T @ a[l], d.sum(axis=0))
        dh = d @ W  # dL/d a_l (the layer's input)
        if l == 0:
            dx = dh
            break
        # a_l = relu(z_{l-1}) (+ a_1 when l == 3, the skip)
        if l == 3:
            dskip = dh  # flows to a_1 = relu(z_0)
        if l == 1 and dskip is not None:
            dh = dh + dskip
        d = dh * (z[l - 1] > 0.0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return flat, dx


def gram_schmidt(a1, a2):
    """Rotation with columns b1 = a1/|a1|, b2 = normalised a2 - (b1.a2) b1, b3 = b1 x b2."""
    b1 = a1 / np.linalg.norm(a1)
    u2 = a2 - np.dot(b1, a2) * b1
    b2 = u2 / np.linalg.norm(u2)
    b3 = np.cross(b1, b2)
    return np.stack([b1, b2, b3], axis=1)


def gram_schmidt_vjp(a1, a2, dR):
    """Derivatives of <dR, phi(a1, a2)> with respect to a1 and a2 (the chain rule of the three
    steps of gram_schmidt written out)."""
    n1 = np.linalg.norm(a1)
    b1 = a1 / n1
    c = np.dot(b1, a2)
    u2 = a2 - c * b1
    n2 = np.linalg.norm(u2)
    b2 = u2 / n2
    g1, g2, g3 = dR[:, 0], dR[:, 1], dR[:, 2]
    # b3 = b1 x b2
    g1 = g1 + np.cross(b2, g3)
    g2 = g2 + np.cross(g3, b1)
    # b2 = u2 / n2
    gu2 = (g2 - np.dot(g2, b2) * b2) / n2
    # u2 = a2 - (b1 . a2) b1
    ga2 = gu2 - np.dot(gu2, b1) * b1
    g1 = g1 - np.dot(gu2, b1) * a2 - c * gu2
    # b1 = a1 / n1
    ga1 = (g1 - np.dot(g1, b1) * b1) / n1
    return ga1, ga2


def unit_scale(P0):
    """RMS distance of the camera centres c = -R^T t from their centroid (1 if they coincide)."""
    P = np.asarray(P0, dtype=np.float64).reshape(-1, 3, 4)
    C = -np.einsum("vji,vj->vi", P[:, :, :3], P[:, :, 3])
    s = float(np.sqrt(((C - C.mean(axis=0)) ** 2).sum(axis=1).mean()))
    return s if s > 0.0 else 1.0


def _tscale(s):
    D = np.ones(12)
    D[3::4] = s
    return D


def poses(theta, delta, P0):
    """P^s (n, 12) of Eq. 3 and the cache for pose_backward."""
    P0 = np.asarray(P0, dtype=np.float64).reshape(-1, 12)
    s = unit_scale(P0)
    D = _tscale(s)
    y, cache = mlp_forward(theta, P0 / D)
    Pp = (P0 + D * y).reshape(-1, 3, 4)
    out = np.zeros((len(P0), 3, 4))
    for v in range(len(P0)):
        out[v, :, :3] = gram_schmidt(Pp[v, :, 0], Pp[v, :, 1])
        out[v, :, 3] = Pp[v, :, 3] + s * np.asarray(delta[v])
    return out.reshape(-1, 12), (cache, Pp, s)


def euclidean_pose_grad(T, G):
    """The objective's derivatives with respect to the entries of each pose [R | t], from its
    left-perturbation gradient G = (g_v, g_w): under T <- Exp(xi) T a change dR = [w]x R,
    dt = [w]x t + v, so dL = g_v . dt + (g_w + g_v x t) . w.  Returns dL/dt = g_v and a dL/dR
    whose tangent part reproduces that (the normal part does not matter: phi only moves R
    along SO(3)): dL/dR = 1/2 [g_w + g_v x t]x R."""
    T = np.asarray(T, dtype=np.float64).reshape(-1, 3, 4)
    G = np.asarray(G, dtype=np.float64).reshape(-1, 6)
    dR = np.zeros((len(T), 3, 3))
    dt = G[:, :3].copy()
    for v in range(len(T)):
        w = G[v, 3:] + np.cross(G[v, :3], T[v, :, 3])
        K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
        dR[v] = 0.5 * K @ T[v, :, :3]
    return dR, dt


def pose_backward(theta, cache, T, G):
    """dL/dtheta and dL/ddelta from the left-perturbation gradient G at the poses T = P^s."""
    mcache, Pp, s = cache
    dR, dt = euclidean_pose_grad(T, G)
    dy = np.zeros((len(Pp), 3, 4))
    for v in range(len(Pp)):
        ga1, ga2 = gram_schmidt_vjp(Pp[v, :, 0], Pp[v, :, 1], dR[v])
        dy[v, :, 0] = ga1
        dy[v, :, 1] = ga2
        dy[v, :, 3] = s * dt[v]
    gtheta, _ = mlp_backward(theta, mcache, dy.reshape(-1, 12))
    return gtheta, s * dt


def lr_at(step, lr_max=3e-3, warmup=25, total=2000):
    """Learning rate of step s (0-based): the k-th warm-up step (k = s + 1 <= warmup) uses
    k / warmup of lr_max; afterwards cosine decay from lr_max at s = warmup - 1 to 0 at
    s = total - 1 (held at 0 beyond)."""
    if step < warmup:
        return lr_max * (step + 1) / warmup
    span = max(total - warmup, 1)
    t = min(step - warmup + 1, span) / span
    return lr_max * 0.5 * (1.0 + np.cos(np.pi * t))


def adamw(p, g, m, v, step, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW step (decoupled weight decay, scaled by the step's learning rate), in place."""
    m *= beta1
    m += (1.0 - beta1) * g
    v *= beta2
    v += (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** (step + 1))
    vh = v / (1.0 - beta2 ** (step + 1))
    p *= 1.0 - lr * wd
    p -= lr * mh / (np.sqrt(vh) + eps)


class PoseMLP:
    """State of one scene's pose MLP run: parameters, offsets, AdamW moments, step."""

    def __init__(self, theta, P0, wd=0.01, wd_delta=0.1, lr_max=3e-3, warmup=25, total=2000):
        self.theta = np.asarray(theta, dtype=np.float64).copy()
        self.P0 = np.asarray(P0, dtype=np.float64).reshape(-1, 12).copy()
        n = len(self.P0)
        self.delta = np.zeros((n, 3))
        self.m, self.v = np.zeros_like(self.theta), np.zeros_like(self.theta)
        self.md, self.vd = np.zeros((n, 3)), np.zeros((n, 3))
        self.step = 0
        self.wd, self.wd_delta = wd, wd_delta
        self.sched = (lr_max, warmup, total)

    def poses(self):
        return poses(self.theta, self.delta, self.P0)[0]

    def step_with(self, objective):
        """One step: P^s, the objective's loss and left-perturbation gradient there (a callable
        T -> (loss, G) over all views: the shared MLP moves every pose, so no view is frozen),
        the chain rule to theta and delta, AdamW."""
        T, cache = poses(self.theta, self.delta, self.P0)
        loss, G = objective(T)
        G = np.asarray(G, dtype=np.float64).reshape(-1, 6)
        gt, gd = pose_backward(self.theta, cache, T, G)
        lr = lr_at(self.step, *self.sched)
        adamw(self.theta, gt, self.m, self.v, self.step, lr, self.wd)
        adamw(self.delta, gd, self.md, self.vd, self.step, lr, self.wd_delta)
        self.step += 1
        return loss, T
