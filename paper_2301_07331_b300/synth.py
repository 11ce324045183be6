"""Seeded synthetic sky catalogues shaped like HLC2's workloads.

The paper evaluates on survey extracts (SDSS, 2MASS, Gaia; Table 2) that are
not available here.  These generators stand in for them with the same shapes:
small patches, full-sky galactic-plane densities, dense Plummer clusters,
cone pairs and a bulge.  They hold none of the cross-match arithmetic: they
only draw positions, and both the CUDA library and the CPU oracle consume
their output unchanged.

Randomness is counter based -- splitmix64 of (seed, stream, index) -- so every
value depends only on its counter, not on the device, chunking or thread
count.  Everything is written with torch tensor operations and runs on CPU or
CUDA tensors alike.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

_M64 = (1 << 64) - 1


def _s64(v: int) -> int:
    """Python int in [0, 2^64) -> the int64 with the same bits."""
    v &= _M64
    return v - (1 << 64) if v >= (1 << 63) else v


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_MUL1 = _s64(0xBF58476D1CE4E5B9)
_MUL2 = _s64(0x94D049BB133111EB)


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def mix64(x: torch.Tensor) -> torch.Tensor:
    """splitmix64 output function (a bijection of 64-bit patterns)."""
    z = x
    z = (z ^ _srl(z, 30)) * _MUL1
    z = (z ^ _srl(z, 27)) * _MUL2
    return z ^ _srl(z, 31)


def _counters(seed: int, stream: int, n: int, offset: int, device) -> torch.Tensor:
    base = mix64(torch.tensor([_s64(seed * 0x100000001B3 + stream)], dtype=torch.int64))
    idx = torch.arange(offset, offset + n, dtype=torch.int64, device=device)
    return (idx + 1) * _GOLDEN + base.to(device)


def uniform(seed: int, stream: int, n: int, device="cpu", offset: int = 0) -> torch.Tensor:
    """n doubles uniform on [0, 1), 53 random bits each."""
    z = mix64(_counters(seed, stream, n, offset, device))
    return _srl(z, 11).to(torch.float64) * (2.0 ** -53)


def ids(seed: int, stream: int, n: int, device="cpu", offset: int = 0) -> torch.Tensor:
    """n distinct uint64 ids (returned as int64 bit patterns): a bijective
    mix of the running index, so ids never collide within one stream."""
    base = int(mix64(torch.tensor([_s64(seed * 31 + stream)], dtype=torch.int64)))
    idx = torch.arange(offset, offset + n, dtype=torch.int64, device=device)
    return mix64(idx + base)


# ---------------------------------------------------------------------------
# Geometry helpers (float64, radians inside, degrees at the interface).
# ---------------------------------------------------------------------------

_D2R = math.pi / 180.0
_R2D = 180.0 / math.pi


def _wrap360(a: torch.Tensor) -> torch.Tensor:
    a = torch.remainder(a, 360.0)
    return torch.where(a >= 360.0, a - 360.0, a)


def offset_point(ra, dec, bearing_rad, dist_rad):
    """Exact spherical destination: start at (ra, dec) degrees, walk dist_rad
    along the great circle with position angle bearing_rad (north through
    east)."""
    d0 = dec * _D2R
    sd, cd = torch.sin(d0), torch.cos(d0)
    sr, cr = torch.sin(dist_rad), torch.cos(dist_rad)
    sin_d1 = (sd * cr + cd * sr * torch.cos(bearing_rad)).clamp(-1.0, 1.0)
    d1 = torch.asin(sin_d1)
    y = torch.sin(bearing_rad) * sr * cd
    x = cr - sd * sin_d1
    ra1 = ra + torch.atan2(y, x) * _R2D
    return _wrap360(ra1), (d1 * _R2D).clamp(-90.0, 90.0)


# J2000 galactic frame: north galactic pole and the galactic longitude of the
# north celestial pole (IAU 1958 definition transformed to J2000).
_RA_NGP = 192.85948
_DEC_NGP = 27.12825
_L_NCP = 122.93192


def gal2eq(l_deg, b_deg):
    b = b_deg * _D2R
    dl = (_L_NCP - l_deg) * _D2R
    dn = _DEC_NGP * _D2R
    sin_dec = (math.sin(dn) * torch.sin(b) + math.cos(dn) * torch.cos(b) * torch.cos(dl)).clamp(-1, 1)
    dec = torch.asin(sin_dec)
    y = torch.cos(b) * torch.sin(dl)
    x = math.cos(dn) * torch.sin(b) - math.sin(dn) * torch.cos(b) * torch.cos(dl)
    ra = _RA_NGP + torch.atan2(y, x) * _R2D
    return _wrap360(ra), (dec * _R2D).clamp(-90.0, 90.0)


# ---------------------------------------------------------------------------
# Position recipes.
# ---------------------------------------------------------------------------

def sphere_uniform(seed, stream, n, device="cpu", offset=0):
    """Uniform per unit solid angle: ra ~ U[0,360), sin(dec) ~ U[-1,1]."""
    u = uniform(seed, 2 * stream, n, device, offset)
    v = uniform(seed, 2 * stream + 1, n, device, offset)
    ra = _wrap360(u * 360.0)
    dec = torch.asin((2.0 * v - 1.0).clamp(-1, 1)) * _R2D
    return ra, dec


def patch_uniform(seed, stream, n, ra0, ra1, dec0, dec1, device="cpu", offset=0):
    """Uniform per unit solid angle inside an RA/Dec rectangle."""
    u = uniform(seed, 2 * stream, n, device, offset)
    v = uniform(seed, 2 * stream + 1, n, device, offset)
    s0, s1 = math.sin(dec0 * _D2R), math.sin(dec1 * _D2R)
    ra = ra0 + (ra1 - ra0) * u
    dec = (torch.asin((s0 + (s1 - s0) * v).clamp(-1, 1)) * _R2D).clamp(dec0, dec1)
    return _wrap360(ra), dec


def galactic_disk(seed, stream, n, h_deg=10.0, device="cpu", offset=0):
    """Density per unit solid angle proportional to exp(-|b|/h): b drawn from
    pdf ~ exp(-|b|/h) cos(b) by rejection from a truncated exponential, l
    uniform.  Counter slots are fixed (8 candidates per source), so the draw
    of source i does not depend on how many sources are generated."""
    K = 8
    h = h_deg * _D2R
    cap = 1.0 - math.exp(-(math.pi / 2) / h)
    # K candidates per source, from counter slots offset*K .. (offset+n)*K
    uu = uniform(seed, 4 * stream, n * K, device, offset * K).view(n, K)
    vv = uniform(seed, 4 * stream + 1, n * K, device, offset * K).view(n, K)
    cand = -h * torch.log1p(-uu * cap)  # truncated exponential on [0, pi/2)
    acc = vv < torch.cos(cand)
    first = torch.where(acc.any(1), acc.to(torch.int8).argmax(1), torch.full((n,), K - 1, device=device))
    b = cand.gather(1, first.view(-1, 1)).view(-1)
    sgn = uniform(seed, 4 * stream + 2, n, device, offset) < 0.5
    b = torch.where(sgn, -b, b)
    l = uniform(seed, 4 * stream + 3, n, device, offset) * 360.0
    return gal2eq(l, b * _R2D)


def gaussian_blob(seed, stream, n, l0, b0, sigma_deg, device="cpu", offset=0):
    """2D Gaussian of width sigma around (l0, b0) galactic: Rayleigh radius,
    uniform position angle, exact spherical offset."""
    u = uniform(seed, 2 * stream, n, device, offset)
    v = uniform(seed, 2 * stream + 1, n, device, offset)
    rho = sigma_deg * _D2R * torch.sqrt(-2.0 * torch.log1p(-u))
    pa = 2.0 * math.pi * v
    ra0, dec0 = gal2eq(torch.tensor([float(l0)], dtype=torch.float64, device=device),
                       torch.tensor([float(b0)], dtype=torch.float64, device=device))
    return offset_point(ra0.expand(n), dec0.expand(n), pa, rho)


def jitter(seed, stream, ra, dec, sigma_arcsec, device=None, offset=0):
    """Isotropic Gaussian position error: Rayleigh(sigma) distance, uniform
    position angle, applied as an exact spherical offset."""
    n = ra.numel()
    dev = ra.device if device is None else device
    u = uniform(seed, 2 * stream, n, dev, offset)
    v = uniform(seed, 2 * stream + 1, n, dev, offset)
    rho = (sigma_arcsec / 3600.0) * _D2R * torch.sqrt(-2.0 * torch.log1p(-u))
    return offset_point(ra, dec, 2.0 * math.pi * v, rho)


def plummer(seed, stream, n, ra_c, dec_c, a_arcmin, device="cpu", offset=0):
    """Projected Plummer profile around (ra_c, dec_c): R = a sqrt(u/(1-u)),
    u ~ U[0, 0.999)."""
    u = uniform(seed, 2 * stream, n, device, offset) * 0.999
    v = uniform(seed, 2 * stream + 1, n, device, offset)
    R = (a_arcmin / 60.0) * _D2R * torch.sqrt(u / (1.0 - u))
    rc = torch.as_tensor(ra_c, dtype=torch.float64, device=device).expand(n)
    dc = torch.as_tensor(dec_c, dtype=torch.float64, device=device).expand(n)
    return offset_point(rc, dc, 2.0 * math.pi * v, R)


def cone_uniform(seed, stream, n, ra_c, dec_c, radius_deg, device="cpu", offset=0):
    """Uniform per unit solid angle inside a spherical cap."""
    u = uniform(seed, 2 * stream, n, device, offset)
    v = uniform(seed, 2 * stream + 1, n, device, offset)
    cmin = math.cos(radius_deg * _D2R)
    rho = torch.acos((1.0 - u * (1.0 - cmin)).clamp(-1, 1))
    rc = torch.as_tensor(ra_c, dtype=torch.float64, device=device).expand(n)
    dc = torch.as_tensor(dec_c, dtype=torch.float64, device=device).expand(n)
    return offset_point(rc, dc, 2.0 * math.pi * v, rho)


# ---------------------------------------------------------------------------
# Catalogues and the workload configurations.
# ---------------------------------------------------------------------------

@dataclass
class Catalogue:
    ra: torch.Tensor   # float64 degrees
    dec: torch.Tensor  # float64 degrees
    id: torch.Tensor   # int64 bit patterns of uint64 ids

    @property
    def n(self) -> int:
        return int(self.ra.numel())

    def to(self, device) -> "Catalogue":
        return Catalogue(self.ra.to(device), self.dec.to(device), self.id.to(device))

    def numpy(self):
        return (self.ra.cpu().numpy(), self.dec.cpu().numpy(),
                self.id.cpu().numpy().view("uint64"))


def error_radii(seed, stream, n, lo_arcsec=0.05, hi_arcsec=0.4, device="cpu", offset=0):
    """n per-source position error radii in arcsec, log-uniform on [lo, hi]:
    the spread of positional errors inside one survey catalogue, one value
    per source as Eq. 4 takes them."""
    u = uniform(seed, 900 + stream, n, device, offset)
    return lo_arcsec * torch.pow(torch.tensor(hi_arcsec / lo_arcsec, dtype=torch.float64,
                                              device=u.device), u)


def _mixture_galactic(seed, stream, n, frac_uniform, device):
    """frac_uniform of the sources uniform on the sphere, the rest in the
    exp(-|b|/10 deg) disk; the component of source i is drawn per source."""
    sel = uniform(seed, 100 + stream, n, device) < frac_uniform
    ra_u, dec_u = sphere_uniform(seed, 200 + stream, n, device)
    ra_d, dec_d = galactic_disk(seed, 300 + stream, n, 10.0, device)
    return torch.where(sel, ra_u, ra_d), torch.where(sel, dec_u, dec_d)


def _cross_pair(seed, A: Catalogue, nb, frac_jit, sigma_arcsec, fresh_fn, device):
    """Catalogue B: frac_jit of it are jittered copies of the first A sources,
    the rest fresh draws from fresh_fn."""
    nj = int(round(nb * frac_jit))
    ra_j, dec_j = jitter(seed, 500, A.ra[:nj], A.dec[:nj], sigma_arcsec)
    ra_f, dec_f = fresh_fn(nb - nj)
    ra = torch.cat([ra_j, ra_f])
    dec = torch.cat([dec_j, dec_f])
    return Catalogue(ra, dec, ids(seed, 2, nb, device))


def patch_pair(seed=2301073310, na=20000, nb=20000, device="cpu"):
    """A uniform in RA 150-160, Dec 0-10 deg; B = 70% jittered (0.3") copies
    of A plus 30% fresh uniform (not clipped to the patch)."""
    ra, dec = patch_uniform(seed, 1, na, 150.0, 160.0, 0.0, 10.0, device)
    A = Catalogue(ra, dec, ids(seed, 1, na, device))
    B = _cross_pair(seed, A, nb, 0.7, 0.3,
                    lambda m: patch_uniform(seed, 7, m, 150.0, 160.0, 0.0, 10.0, device),
                    device)
    return A, B


def fullsky_pair(seed=2301073311, na=10_000_000, nb=10_000_000, device="cpu"):
    """Full sky, 40% uniform + 60% galactic disk exp(-|b|/10 deg); B = 60%
    jittered (0.5") copies of A plus 40% fresh from the same mixture."""
    ra, dec = _mixture_galactic(seed, 1, na, 0.4, device)
    A = Catalogue(ra, dec, ids(seed, 1, na, device))
    B = _cross_pair(seed, A, nb, 0.6, 0.5,
                    lambda m: _mixture_galactic(seed, 7, m, 0.4, device), device)
    return A, B


def clustered_pair(seed=2301073312, na=400_000_000, nb=300_000_000,
                   n_clusters=200, members=50_000, device="cpu"):
    """The full-sky mixture plus n_clusters Plummer clusters (a = 2') of
    `members` A sources each; B = 60% jittered copies of A + 40% fresh."""
    n_cl = n_clusters * members
    nf = na - n_cl
    ra_f, dec_f = _mixture_galactic(seed, 1, nf, 0.4, device)
    rc, dc = _mixture_galactic(seed, 11, n_clusters, 0.4, device)
    ras, decs = [ra_f], [dec_f]
    for c in range(n_clusters):
        r_, d_ = plummer(seed, 1000 + c, members, rc[c], dc[c], 2.0, device)
        ras.append(r_)
        decs.append(d_)
    A = Catalogue(torch.cat(ras), torch.cat(decs), ids(seed, 1, na, device))
    # jitter an even spread of A (indices floor(i * na / nj), covering the
    # clusters at the end of A too) so that clusters get counterparts
    nj = int(round(nb * 0.6))
    src = (torch.arange(0, nj, device=device, dtype=torch.int64) * na) // nj
    ra_j, dec_j = jitter(seed, 500, A.ra[src], A.dec[src], 0.5)
    ra_x, dec_x = _mixture_galactic(seed, 7, nb - nj, 0.4, device)
    B = Catalogue(torch.cat([ra_j, ra_x]), torch.cat([dec_j, dec_x]), ids(seed, 2, nb, device))
    return A, B


@dataclass
class ConeJob:
    A: Catalogue
    B: Catalogue
    r_arcsec: float
    order: int
    ra_c: float
    dec_c: float
    cone_deg: float


def cone_jobs(seed=2301073313, n_jobs=4096, nmin=1_000, nmax=1_000_000,
              scale=1.0, device="cpu"):
    """n_jobs independent cone pairs: centre uniform on the sphere, cone
    radius U[0.1, 2] deg, N_A and N_B log-uniform on [nmin, nmax] (times
    `scale`), match radius U[0.5, 5] arcsec, uniform density in the cone.
    The order of each job is left at 0 for the caller to choose."""
    u = uniform(seed, 1, n_jobs * 6).view(n_jobs, 6)
    jobs = []
    lo, hi = math.log(nmin), math.log(nmax)
    for j in range(n_jobs):
        ra_c = float(u[j, 0]) * 360.0
        dec_c = math.degrees(math.asin(2.0 * float(u[j, 1]) - 1.0))
        cone = 0.1 + 1.9 * float(u[j, 2])
        na = max(1, int(round(math.exp(lo + (hi - lo) * float(u[j, 3])) * scale)))
        nb = max(1, int(round(math.exp(lo + (hi - lo) * float(u[j, 4])) * scale)))
        r = 0.5 + 4.5 * float(u[j, 5])
        ra, dec = cone_uniform(seed, 10 + 4 * j, na, ra_c, dec_c, cone, device)
        A = Catalogue(ra, dec, ids(seed, 10 + 4 * j, na, device))
        ra, dec = cone_uniform(seed, 12 + 4 * j, nb, ra_c, dec_c, cone, device)
        B = Catalogue(ra, dec, ids(seed, 12 + 4 * j, nb, device))
        jobs.append(ConeJob(A, B, r, 0, ra_c, dec_c, cone))
    return jobs


def bulge_pair(seed=2301073314, na=500_000_000, nb=500_000_000, device="cpu"):
    """Density spanning ~1e2 to ~1e6 per sq deg: 0.825% uniform, 67.8%
    galactic disk, 31.4% bulge (2D Gaussian sigma 5 deg at l = b = 0);
    B = 60% jittered copies of A + 40% fresh."""
    def draw(stream, n):
        c = uniform(seed, 100 + stream, n, device)
        ra_u, dec_u = sphere_uniform(seed, 200 + stream, n, device)
        ra_d, dec_d = galactic_disk(seed, 300 + stream, n, 10.0, device)
        ra_b, dec_b = gaussian_blob(seed, 400 + stream, n, 0.0, 0.0, 5.0, device)
        ra = torch.where(c < 0.00825, ra_u, torch.where(c < 0.00825 + 0.678, ra_d, ra_b))
        dec = torch.where(c < 0.00825, dec_u, torch.where(c < 0.00825 + 0.678, dec_d, dec_b))
        return ra, dec
    ra, dec = draw(1, na)
    A = Catalogue(ra, dec, ids(seed, 1, na, device))
    B = _cross_pair(seed, A, nb, 0.6, 0.5, lambda m: draw(7, m), device)
    return A, B
