"""Oracle backend of paper_1905_05524_gb300.exchange.StripStepper (test
infrastructure): one rank's strip advanced by the oracle, edge face data
packed as [nx, 8, n] tensors (q-bar and normal flux)."""
import torch

from oracle.aderdg import Mesh, Solver


class OracleStrip:
    def __init__(self, params, nx, rows, first_row, ny_global, Lx, Ly, y0, bc_y, u):
        hy = Ly / ny_global
        self.s = Solver(Mesh(nx, rows, x0=0.0, y0=y0 + first_row * hy, Lx=Lx, Ly=rows * hy,
                             bc_x="periodic" if bc_y.startswith("halo") or bc_y == "periodic" else "wall",
                             bc_y=bc_y), params)
        self.nx, self.rows = nx, rows
        self.u = u

    def predictor(self, dt):
        self.dt = dt
        _, self.tavg = self.s.predictor(self.u, dt)
        self.tr = self.s.face_traces(self.tavg)

    def boundary_traces(self):
        n = self.nx
        south = torch.cat([self.tr["S"]["q"][:n], self.tr["S"]["f"][:n]], 1).contiguous()
        north = torch.cat([self.tr["N"]["q"][-n:], self.tr["N"]["f"][-n:]], 1).contiguous()
        return south, north

    def set_halo(self, south, north):
        self.halo = {"S": (south[:, :4], south[:, 4:]) if south is not None else None,
                     "N": (north[:, :4], north[:, 4:]) if north is not None else None}

    def corrector(self, dt):
        self.u = self.s.corrector(self.u, dt, self.tavg, self.halo)
