"""Discrete velocity sets (oracle copy; test infrastructure only).

D3Q19 directions, ordering and weights follow the paper's D3Q19 table (§3).
D2Q5 and D3Q7 are the textbook minimal advection-diffusion sets: w_0 = 1/3,
w_{1..4} = 1/6 with c_s^2 = 1/3 (D2Q5) and w_0 = 1/4, w_{1..6} = 1/8 with
c_s^2 = 1/4 (D3Q7); for both, sum_k w_k e_k e_k = c_s^2 I.
Vectors are (x, y, z); 2D sets have z = 0.
"""
from dataclasses import dataclass
import torch


@dataclass(frozen=True)
class Lattice:
    name: str
    e: tuple        # Q integer vectors (x, y, z)
    w: tuple        # Q weights
    cs2: float      # squared lattice sound speed

    @property
    def Q(self):
        return len(self.w)

    def e_tensor(self):
        return torch.tensor(self.e, dtype=torch.float64)

    def w_tensor(self):
        return torch.tensor(self.w, dtype=torch.float64)

    def opposite(self, k):
        """Index of the direction -e_k."""
        ek = self.e[k]
        for j, ej in enumerate(self.e):
            if ej == (-ek[0], -ek[1], -ek[2]):
                return j
        raise ValueError("lattice is not symmetric")


D2Q5 = Lattice("D2Q5",
               e=((0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0)),
               w=(1 / 3, 1 / 6, 1 / 6, 1 / 6, 1 / 6), cs2=1 / 3)

D3Q7 = Lattice("D3Q7",
               e=((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)),
               w=(1 / 4,) + (1 / 8,) * 6, cs2=1 / 4)

# §3, D3Q19 table: k = 0; 1..6 axis directions (w = 1/18); 7..18 face diagonals (w = 1/36)
D3Q19 = Lattice("D3Q19",
                e=((0, 0, 0),
                   (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                   (1, 1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, -1), (0, 1, 1), (0, -1, -1),
                   (1, -1, 0), (-1, 1, 0), (1, 0, -1), (-1, 0, 1), (0, 1, -1), (0, -1, 1)),
                w=(1 / 3,) + (1 / 18,) * 6 + (1 / 36,) * 12, cs2=1 / 3)

# §3, D2Q9 table, in the table's order (the 2D ripening workload's lattice for g, h^A, h^B)
D2Q9 = Lattice("D2Q9",
               e=((0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
                  (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)),
               w=(4 / 9,) + (1 / 9,) * 4 + (1 / 36,) * 4, cs2=1 / 3)

BY_NAME = {"D2Q5": D2Q5, "D3Q7": D3Q7, "D3Q19": D3Q19, "D2Q9": D2Q9}
